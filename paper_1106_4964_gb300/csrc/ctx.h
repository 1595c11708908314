// Library context (host side) shared by the API and solver translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/overlap.h"
#include "ov_internal.cuh"
#include "ov_kernels.h"

struct ov_field {
    ov::FieldDesc d;
    ov_ctx* owner;
};

namespace ov {

// workspace slots (internal fields cached per (slot, prec, nrhs))
// device scalar scratch (c->dscal, doubles): coefficient blocks, then CG scalars
constexpr int DSCAL_DOUBLES = 65536;
constexpr int DSCAL_COEF = 57344;   // [0, DSCAL_COEF): coefficient blocks (double2 pairs)
constexpr int DSCAL_CGCO = 57344;   // double2 [K][R] per-rhs coefficients
constexpr int DSCAL_CHCO = 59392;   // double2 [3][R] chiral-sector operator, [2][R] sector projection
constexpr int DSCAL_NORM = 61440;   // per-rhs norms
constexpr int DSCAL_DOT = 62464;    // per-rhs dots (double2)
constexpr int DSCAL_TMP = 64512;    // single-value scratch

enum Slot {
    WS_IN = 0, WS_OUT, WS_PH, WS_W, WS_T, WS_B0, WS_B1, WS_B2,
    WS_CG_X, WS_CG_R, WS_CG_P, WS_CG_Q, WS_CG_Z, WS_CG_B, WS_CG_T, WS_CG_U, WS_CG_RS, WS_CG_PS, WS_CG_QS, WS_CG_XS,
    WS_CG_BH, WS_CG_XH, WS_TC0, WS_TC1, WS_MX0, WS_MX1, WS_RS, WS_RR, WS_RP, WS_RQ, WS_RT,
    WS_LZ_W, WS_LZ_WB, WS_LZ_T, WS_LZ_F0, WS_LZ_F1, WS_LZ_F2, WS_LZ_F3, WS_NET_S, WS_NET_H, WS_NET_G, WS_NET_GH, WS_AUX0, WS_AUX1,
    WS_COUNT
};

struct EigSet {
    int nev = 0;
    std::vector<double> vals;   // host copy
    FieldDesc vec[NPREC] = {};      // per storage precision (F64 is the master copy)
    double* d_sign = nullptr;   // device sign(lam_i) (which = 0)
    void* tc_rows = nullptr;    // bf16 rows of the tensor-core projection [nev][24V]
    size_t tc_bytes = 0;
    void* tc_lo = nullptr;      // bf16 remainders of the FP32 copy (FP32-class tensor-core operand)
    size_t tc_lo_bytes = 0;
};

struct NetState;  // learned preconditioner (net.cu)

}  // namespace ov

struct ov_ctx {
    int dims[4];
    double bc[4];
    ov::Geom g;
    int device = 0;
    long long bytes = 0;

    void* gauge[ov::NPREC] = {};
    bool have_gauge = false;

    double rho = 1.5, eps = 0.05, lmax = 0.0;
    int degree = 0;
    std::vector<double> coef;
    // rational sign (Eq. 12): sign_backend 1 uses P(x) = sum_i rb_i / (x + rc_i) by multi-shift CG
    int sign_backend = 0;
    std::vector<double> rb, rc;
    double rdelta = 0.0;
    int rational_pass = 2;        // 1 single pass (2n shifted vectors), 2 double pass (scalars, then one sum)
    double rational_tol = 1e-12;  // relative residual of every shifted solve
    long long rational_iters = 0; // CG iterations of the last rational sign application (instrumentation)
    // adaptive-precision CG: the inner operator's polynomial (degree_in <= degree, delta <= adaptive_delta)
    double adaptive_delta = 0.0;
    int degree_in = 0;
    std::vector<double> coef_in;
    bool have_poly = false;

    ov::EigSet eig[2];

    std::map<std::tuple<int, int, int>, ov::FieldDesc> ws;
    double* partials = nullptr;
    size_t partials_bytes = 0;
    double* dscal = nullptr;  // device scalar scratch, DSCAL_DOUBLES doubles
    void* stage[2] = {nullptr, nullptr};
    size_t stage_bytes[2] = {0, 0};
    unsigned* derr = nullptr;

    std::map<std::pair<int, int>, std::tuple<int, int, int>> shape;  // (prec, nrhs) -> (bx, by, variant)

    ov::NetState* net = nullptr;

    // captured CUDA graphs of whole operator applications:
    // key (kind, in, out, prec, nrhs, mass, g5) -> (executable graph, dslash launches inside)
    std::map<std::tuple<int, const void*, const void*, int, int, double, int>, std::pair<cudaGraphExec_t, long long>>
        graphs;
    bool use_graphs = true;
    long long graph_captures = 0, graph_replays = 0;  // instrumentation (ov_graph_stats)
    // library-owned stream (and its two ordering events) on which graphs run for callers that pass the
    // legacy default stream, which cannot be captured
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};

    // instrumentation: number of dslash launches issued through this context
    long long dslash_launches = 0;

    // solver options (ov_set_option)
    double reliable_delta = 0.1;  // FP64 true residual when the sloppy residual drops by this factor
    int filter_hw = 100;          // Chebyshev filter degree on H_w^2 (deflate which = 0)
    int filter_dd = 8;            // Chebyshev filter degree on D^dag D (deflate which = 1)
    int eig_prec = -1;            // operator precision inside deflate: -1 automatic, else ov_prec
    int proj_tc = 1;              // 16-bit overlap: low-mode projection on the tensor cores
    int net_sym = 1;              // learned preconditioner applied as (M + M^dag) / 2
    int hi_prec = ov::P_F64;      // accurate arithmetic of the solvers: P_F64 or P_DF64
    int chiral = 0;               // ov_cg_solve: inner operator restricted to one chiral sector
    int clenshaw_f32 = 1;         // 16-bit overlap: FP32 work vectors in the Clenshaw recurrence
    long long wait_polls = ov::DSLASH_WAIT_POLLS;  // first bounded wait of the bulk-copy dslash (option "wait_polls")

    // tensor-core projection buffers (proj_tc.cu)
    void* tc_b = nullptr;
    size_t tc_b_bytes = 0;
    void* tc_cb = nullptr;  // bf16 coefficient operand of the tensor-core V c update
    size_t tc_cb_bytes = 0;
    void* rcoef = nullptr;  // device coefficient blocks of the rational sign's multi-shift CG
    size_t rcoef_bytes = 0;
    int* tc_err = nullptr;

    std::string err;
};

namespace ov {

int set_err(ov_ctx* c, int code, const char* fmt, ...);
#define OV_CUDA(ctx, call)                                                                         \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return ov::set_err(ctx, e_ == cudaErrorMemoryAllocation ? OV_ENOMEM : OV_ECUDA,        \
                               "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)
#define OV_TRY(x)                 \
    do {                          \
        int s_ = (x);             \
        if (s_ != OV_OK) return s_; \
    } while (0)

int dev_alloc(ov_ctx* c, void** p, size_t bytes);
void graphs_clear(ov_ctx* c);
void dev_free(ov_ctx* c, void* p, size_t bytes);
int field_alloc(ov_ctx* c, int prec, int nrhs, FieldDesc* f);
void field_free(ov_ctx* c, FieldDesc* f);
int ws_field(ov_ctx* c, int slot, int prec, int nrhs, FieldDesc* f);
void ws_release(ov_ctx* c, int slot, int prec = -1, int nrhs = -1);
int ensure_partials(ov_ctx* c, size_t bytes);
bool is_device_ptr(const void* p);
int stage_in(ov_ctx* c, int which, const void* src, size_t bytes, cudaStream_t st, const double** dev);
int stage_out_buffer(ov_ctx* c, int which, void* dst, size_t bytes, double** dev);
int stage_out_finish(ov_ctx* c, void* dst, const double* dev, size_t bytes, cudaStream_t st);
int gauge_prec_for(int prec);
int check_kernel_flags(ov_ctx* c, cudaStream_t st);
// progress lines of the iterative solvers on stderr when the environment sets OV_VERBOSE=1
bool verbose();
int eig_vectors(ov_ctx* c, int which, int prec, cudaStream_t st, FieldDesc* out);

// operators on internal fields
int dslash_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double a, double b, int g5_core, int g5_out,
                 int ny, const FieldDesc* y, const double* sy, cudaStream_t st, int gprec = -1);
int overlap_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, cudaStream_t st);
// out = gamma5^g5_out D(m) in (graph-captured like overlap_apply)
int overlap_g5_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, int g5_out, cudaStream_t st);
// out = D(m)^dag D(m) in; poly 1: with the inner polynomial of the adaptive-precision CG
int normal_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, cudaStream_t st, int poly = 0);
int chiral_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, const double2* dcoef,
                 cudaStream_t st, int poly = 0);
int chiral_setup(ov_ctx* c, const FieldDesc& f, const FieldDesc& tmp, double mass, cudaStream_t st);

// level-1 helpers (stream-ordered); results of reductions land in device memory
int lincomb(ov_ctx* c, const FieldDesc& out, int K, const FieldDesc* x, const double2* hcoef, const double2* dcoef,
            int g5mask, double* dnorm_out, cudaStream_t st);
int dot(ov_ctx* c, const FieldDesc& x, const FieldDesc& y, double2* dout, cudaStream_t st);
int norm2(ov_ctx* c, const FieldDesc& x, double* dout, cudaStream_t st);
int convert(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, cudaStream_t st);
int copy_field(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, cudaStream_t st);

// s = sum_i b_i (Q^2 + c_i)^-1 src, the rational P(Q^2) of Eq. 12 (solver.cu); gprec: link precision
int rational_solve(ov_ctx* c, const FieldDesc& src, const FieldDesc& s, int gprec, cudaStream_t st);
// solvers (solver.cu)
int estimate_lambda_max(ov_ctx* c, int steps, double* lmax, cudaStream_t st);
int deflate_impl(ov_ctx* c, int which, int nev, double tol, cudaStream_t st);
// warm: x holds the starting iterate (else the solve starts from x = 0)
int cg_impl(ov_ctx* c, const FieldDesc& b, const FieldDesc& x, double mass, double tol, int max_iter, int precond,
            int inner_prec, ov_solve_info* info, cudaStream_t st, bool warm = false);
// one multi-shifted CG for several masses, then a per-mass refinement (solver.cu)
int multimass_impl(ov_ctx* c, const FieldDesc& b, const FieldDesc* x, int nmass, const double* masses, double tol,
                   int max_iter, int inner_prec, int output, ov_solve_info* info, cudaStream_t st);
void net_free(ov_ctx* c);

// eigenpairs
void eig_clear(ov_ctx* c, EigSet& E);
// tensor-core projection (proj_tc.cu): c[i][r] = eta_i^dag psi_r, device double2 [nev][R]
// nsplit 1: bf16 rows and bf16 psi; 2: plus the bf16 remainders of both (FP32-class coefficients)
int proj_dots_tc(ov_ctx* c, int which, const FieldDesc& psi, double2* cout, cudaStream_t st, int nsplit = 1);
int proj_tc_status(ov_ctx* c, cudaStream_t st);
// out1 = psi - sum_i eta_i c_i, out2 = gamma5 sum_i s_i c_i eta_i on the tensor cores (FP32 / 16-bit fields)
int proj_update_tc(ov_ctx* c, int which, const FieldDesc& psi, const double2* dcoef, const double* dsign,
                   const FieldDesc& out1, const FieldDesc& out2, cudaStream_t st);

}  // namespace ov
