// Host-side launchers of the library's CUDA kernels (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "ov_internal.cuh"

namespace ov {

// ---------------------------------------------------------------- dslash
struct DslashArgs {
    Geom g;
    const char* gauge;           // packed links of the gauge precision
    const char* in;              // input field (all rhs, both parities)
    const float* in_n;
    char* out;
    float* out_n;
    const char* y[3];            // extra epilogue fields (same layout as out)
    const float* y_n[3];
    double a, b;                 // core = a psi(n) + b * sum of hops
    double sy[3];
    float fa, fb, fsy[3];        // the same coefficients for FP32 arithmetic
    int nrhs;
    int g5_core, g5_out;
    unsigned* err;               // set to 1 when a bounded wait of a staged variant times out
    long long wait_polls;        // limit of the bulk-copy variants' first mbarrier wait (polls)
};
constexpr long long DSLASH_WAIT_POLLS = 1ll << 22;  // default first-wait limit (also bounded by 2 s)
// var: 0 unbounded registers, 1 and 2 capped for occupancy, 3 per-thread cp.async staging
// (FP32 math, by = 1), 4 block-wide bulk-copy (TMA) staging of the neighbour ranges (FP32 math;
// fixed 128-site blocks, bx and by ignored), 5 the same with the eight links loaded before the wait,
// 6 and 7: 2 and 4 right-hand sides per thread sharing each link (FP32 math; by counts rhs groups),
// 8 and 9: the loads of 4 or 8 hops issued together before their arithmetic (FP32 math),
// 10 and 11: 2 or 4 right-hand sides per thread as pairs on the packed FP32 pipe (by counts rhs groups)
cudaError_t launch_dslash(const DslashArgs& A, int sp, int gp, int ny, int bx, int by, int var, cudaStream_t st);
// the variant groups, one translation unit each (grid and block already derived from bx, by)
cudaError_t launch_dslash_regs(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block, cudaStream_t st);
cudaError_t launch_dslash_staged(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block,
                                 cudaStream_t st);
cudaError_t launch_dslash_multi(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block, cudaStream_t st);
cudaError_t launch_dslash_batched(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block,
                                  cudaStream_t st);
cudaError_t launch_dslash_pair(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block, cudaStream_t st);
constexpr int DSLASH_VARIANTS = 12;

// ---------------------------------------------------------------- layout conversion
// canonical complex128 [nrhs][V][12] (device) <-> internal field
cudaError_t launch_pack(const Geom& g, const double* canon, const FieldDesc& f, int gamma5, cudaStream_t st);
cudaError_t launch_unpack(const Geom& g, const FieldDesc& f, double* canon, int gamma5, cudaStream_t st);
// canonical complex128 gauge [V][4][3][3] (device) -> reconstruct-12 links in `prec`;
// *dev_err receives max |U U^dag - 1| and max |row2 - conj(row0 x row1)| (as float bits, atomicMax)
cudaError_t launch_pack_gauge(const Geom& g, const double* canon, void* out, int prec, unsigned* dev_err,
                              cudaStream_t st);
// precision conversion between two internal fields of equal nrhs
cudaError_t launch_convert(const Geom& g, const FieldDesc& in, const FieldDesc& out, cudaStream_t st);

// ---------------------------------------------------------------- level-1
// out_r = sum_{j<K} c_j[r] * G_j x_j,r  with complex coefficients (device array [K][nrhs] of double2,
// or uniform host values when dcoef == null), G_j = gamma5 if bit j of g5mask.  Optional fused
// per-rhs |out|^2 partials (FP64) into `partials` ([nrhs][nblk] doubles).
struct LincombArgs {
    int K;
    FieldDesc x[4];
    const double2* dcoef;
    double2 hcoef[4];
    int g5mask;
    FieldDesc out;
    double* partials;  // null: no norm
};
cudaError_t launch_lincomb(const Geom& g, const LincombArgs& A, int nblk, cudaStream_t st);
// per-rhs x^dag y partial sums (complex, FP64) -> partials [nrhs][nblk] double2
cudaError_t launch_dot(const Geom& g, const FieldDesc& x, const FieldDesc& y, double2* partials, int nblk,
                       cudaStream_t st);
// sum the partials of each rhs in fixed order: out[r] = sum_b partials[r][b]; ncomp = 1 (double) or 2 (double2)
cudaError_t launch_finalize(const double* partials, int nblk, int nrhs, int ncomp, double* out, cudaStream_t st);
int reduce_blocks(const Geom& g);
// uniform(-1,1) entries from a counter-based hash of (seed, element)
cudaError_t launch_fill_random(const Geom& g, const FieldDesc& f, unsigned long long seed, cudaStream_t st);

// ---------------------------------------------------------------- deflation projections
// c[i][r] = eta_i^dag psi_r for i < nev (eta: nev fields of 1 rhs, contiguous); partial sums [nblk][nev][nrhs]
cudaError_t launch_proj_dots(const Geom& g, const FieldDesc& eta, int nev, const FieldDesc& psi, double2* partials,
                             int nblk, cudaStream_t st);
cudaError_t launch_proj_finalize(const double2* partials, int nparts, int n, double2* out, cudaStream_t st);
int proj_groups(int nrhs);  // warp groups per block of proj_dots: partial count = nblk * proj_groups
// out1_r = psi_r - sum_i eta_i c[i][r];  out2_r = gamma5 sum_i eta_i s_i c[i][r] (if out2.data)
cudaError_t launch_proj_update(const Geom& g, const FieldDesc& eta, int nev, const double2* c, const double* s,
                               const FieldDesc& psi, const FieldDesc& out1, const FieldDesc& out2, cudaStream_t st);

}  // namespace ov
