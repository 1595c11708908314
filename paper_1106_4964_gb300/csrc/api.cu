// C ABI of the library: context, gauge packing, dslash / H_w / overlap
// application, internal-layout fields.  The solvers (eigensolver, CG) live in
// solver.cu, the learned preconditioner in net.cu.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "ctx.h"

using namespace ov;

namespace ov {

int set_err(ov_ctx* c, int code, const char* fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int dev_alloc(ov_ctx* c, void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return OV_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(c, OV_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    c->bytes += (long long)bytes;
    return OV_OK;
}

void dev_free(ov_ctx* c, void* p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        c->bytes -= (long long)bytes;
    }
}

static size_t data_bytes(int prec, int nrhs, int Vh) { return (size_t)nrhs * 2 * spinor_chunks(prec) * 16 * Vh; }
static size_t norm_bytes(int prec, int nrhs, int Vh) { return has_norm(prec) ? (size_t)nrhs * 2 * Vh * 4 : 0; }

int field_alloc(ov_ctx* c, int prec, int nrhs, FieldDesc* f)
{
    *f = FieldDesc{prec, nrhs, c->g.Vh, nullptr, nullptr};
    void* p = nullptr;
    OV_TRY(dev_alloc(c, &p, data_bytes(prec, nrhs, c->g.Vh)));
    f->data = (char*)p;
    if (has_norm(prec)) {
        void* q = nullptr;
        int s = dev_alloc(c, &q, norm_bytes(prec, nrhs, c->g.Vh));
        if (s != OV_OK) {
            dev_free(c, p, data_bytes(prec, nrhs, c->g.Vh));
            f->data = nullptr;
            return s;
        }
        f->norm = (float*)q;
    }
    return OV_OK;
}

void field_free(ov_ctx* c, FieldDesc* f)
{
    if (f->data) dev_free(c, f->data, data_bytes(f->prec, f->nrhs, f->Vh));
    if (f->norm) dev_free(c, f->norm, norm_bytes(f->prec, f->nrhs, f->Vh));
    f->data = nullptr;
    f->norm = nullptr;
}

int ws_field(ov_ctx* c, int slot, int prec, int nrhs, FieldDesc* f)
{
    auto key = std::make_tuple(slot, prec, nrhs);
    auto it = c->ws.find(key);
    if (it != c->ws.end()) {
        *f = it->second;
        return OV_OK;
    }
    OV_TRY(field_alloc(c, prec, nrhs, f));
    c->ws[key] = *f;
    return OV_OK;
}

// Free every cached work field of `slot` (of precision `prec` and `nrhs` right-hand sides; -1: any).
// Captured graphs may hold their addresses: the caller clears the graphs first.
void ws_release(ov_ctx* c, int slot, int prec, int nrhs)
{
    for (auto it = c->ws.begin(); it != c->ws.end();) {
        const auto& k = it->first;
        if (std::get<0>(k) == slot && (prec < 0 || std::get<1>(k) == prec) && (nrhs < 0 || std::get<2>(k) == nrhs)) {
            field_free(c, &it->second);
            it = c->ws.erase(it);
        } else {
            ++it;
        }
    }
}

int ensure_partials(ov_ctx* c, size_t bytes)
{
    if (bytes <= c->partials_bytes) return OV_OK;
    graphs_clear(c);  // captured graphs hold the old pointer
    // the old buffer may still be read by queued kernels: wait before freeing
    if (c->partials) {
        cudaDeviceSynchronize();
        dev_free(c, c->partials, c->partials_bytes);
    }
    c->partials = nullptr;
    c->partials_bytes = 0;
    void* p = nullptr;
    OV_TRY(dev_alloc(c, &p, bytes));
    c->partials = (double*)p;
    c->partials_bytes = bytes;
    return OV_OK;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int ensure_stage(ov_ctx* c, int which, size_t bytes)
{
    if (bytes <= c->stage_bytes[which]) return OV_OK;
    if (c->stage[which]) {
        cudaDeviceSynchronize();
        dev_free(c, c->stage[which], c->stage_bytes[which]);
    }
    c->stage[which] = nullptr;
    c->stage_bytes[which] = 0;
    OV_TRY(dev_alloc(c, &c->stage[which], bytes));
    c->stage_bytes[which] = bytes;
    return OV_OK;
}

int stage_in(ov_ctx* c, int which, const void* src, size_t bytes, cudaStream_t st, const double** dev)
{
    if (is_device_ptr(src)) {
        *dev = (const double*)src;
        return OV_OK;
    }
    OV_TRY(ensure_stage(c, which, bytes));
    OV_CUDA(c, cudaMemcpyAsync(c->stage[which], src, bytes, cudaMemcpyHostToDevice, st));
    *dev = (const double*)c->stage[which];
    return OV_OK;
}

int stage_out_buffer(ov_ctx* c, int which, void* dst, size_t bytes, double** dev)
{
    if (is_device_ptr(dst)) {
        *dev = (double*)dst;
        return OV_OK;
    }
    OV_TRY(ensure_stage(c, which, bytes));
    *dev = (double*)c->stage[which];
    return OV_OK;
}

int stage_out_finish(ov_ctx* c, void* dst, const double* dev, size_t bytes, cudaStream_t st)
{
    if ((const void*)dev == dst) return OV_OK;
    OV_CUDA(c, cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    return OV_OK;
}

int gauge_prec_for(int prec) { return prec; }

bool verbose()
{
    static const bool v = [] {
        const char* e = std::getenv("OV_VERBOSE");
        return e && e[0] == '1';
    }();
    return v;
}

// Flags set by kernels whose bounded waits ran out (derr[2]); read and cleared.
int check_kernel_flags(ov_ctx* c, cudaStream_t st)
{
    unsigned f = 0;
    OV_CUDA(c, cudaMemcpyAsync(&f, c->derr + 2, sizeof f, cudaMemcpyDeviceToHost, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    if (f) {
        OV_CUDA(c, cudaMemsetAsync(c->derr + 2, 0, sizeof f, st));
        return set_err(c, OV_ETIMEOUT, "a staged dslash launch timed out waiting for its copies");
    }
    return OV_OK;
}

int eig_vectors(ov_ctx* c, int which, int prec, cudaStream_t st, FieldDesc* out)
{
    EigSet& E = c->eig[which];
    if (E.nev == 0) return set_err(c, OV_ESTATE, "no eigenpairs stored (which=%d)", which);
    if (!E.vec[prec].data) {
        OV_TRY(field_alloc(c, prec, E.nev, &E.vec[prec]));
        OV_CUDA(c, launch_convert(c->g, E.vec[P_F64], E.vec[prec], st));
    }
    *out = E.vec[prec];
    return OV_OK;
}

static std::tuple<int, int, int> default_shape(int prec, int nrhs)
{
    if (nrhs == 1) return {wide(prec) ? 64 : 128, 1, 0};
    const int cap = wide(prec) ? 8 : 16;
    int by = nrhs > cap ? cap : nrhs;
    return {32, by, 0};
}

int dslash_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double a, double b, int g5_core, int g5_out,
                 int ny, const FieldDesc* y, const double* sy, cudaStream_t st, int gprec)
{
    if (gprec < 0) gprec = gauge_prec_for(in.prec);
    DslashArgs A;
    memset(&A, 0, sizeof A);
    A.g = c->g;
    A.err = c->derr + 2;
    A.wait_polls = c->wait_polls;
    A.gauge = (const char*)c->gauge[gprec];
    A.in = in.data;
    A.in_n = in.norm;
    A.out = out.data;
    A.out_n = out.norm;
    for (int j = 0; j < ny; ++j) {
        A.y[j] = y[j].data;
        A.y_n[j] = y[j].norm;
        A.sy[j] = sy[j];
        A.fsy[j] = (float)sy[j];
    }
    A.a = a;
    A.b = b;
    A.fa = (float)a;
    A.fb = (float)b;
    A.nrhs = in.nrhs;
    A.g5_core = g5_core;
    A.g5_out = g5_out;
    auto it = c->shape.find({in.prec, in.nrhs});
    std::tuple<int, int, int> sh = it != c->shape.end() ? it->second : default_shape(in.prec, in.nrhs);
    OV_CUDA(c, launch_dslash(A, in.prec, gprec, ny, std::get<0>(sh), std::get<1>(sh), std::get<2>(sh), st));
    c->dslash_launches++;
    return OV_OK;
}

int lincomb(ov_ctx* c, const FieldDesc& out, int K, const FieldDesc* x, const double2* hcoef, const double2* dcoef,
            int g5mask, double* dnorm_out, cudaStream_t st)
{
    LincombArgs A;
    memset(&A, 0, sizeof A);
    A.K = K;
    for (int j = 0; j < K; ++j) {
        A.x[j] = x[j];
        if (hcoef) A.hcoef[j] = hcoef[j];
    }
    A.dcoef = dcoef;
    A.g5mask = g5mask;
    A.out = out;
    const int nblk = reduce_blocks(c->g);
    if (dnorm_out) {
        OV_TRY(ensure_partials(c, (size_t)nblk * out.nrhs * sizeof(double)));
        A.partials = c->partials;
    }
    OV_CUDA(c, launch_lincomb(c->g, A, nblk, st));
    if (dnorm_out) OV_CUDA(c, launch_finalize(c->partials, nblk, out.nrhs, 1, dnorm_out, st));
    return OV_OK;
}

int dot(ov_ctx* c, const FieldDesc& x, const FieldDesc& y, double2* dout, cudaStream_t st)
{
    const int nblk = reduce_blocks(c->g);
    OV_TRY(ensure_partials(c, (size_t)nblk * x.nrhs * sizeof(double2)));
    OV_CUDA(c, launch_dot(c->g, x, y, (double2*)c->partials, nblk, st));
    OV_CUDA(c, launch_finalize(c->partials, nblk, x.nrhs, 2, (double*)dout, st));
    return OV_OK;
}

int norm2(ov_ctx* c, const FieldDesc& x, double* dout2, cudaStream_t st)
{
    // dout2 receives [nrhs] double2 (re = |x|^2)
    return dot(c, x, x, (double2*)dout2, st);
}

int convert(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, cudaStream_t st)
{
    OV_CUDA(c, launch_convert(c->g, in, out, st));
    return OV_OK;
}

int copy_field(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, cudaStream_t st)
{
    if (in.prec != out.prec) return convert(c, in, out, st);
    OV_CUDA(c, cudaMemcpyAsync(out.data, in.data, data_bytes(in.prec, in.nrhs, in.Vh), cudaMemcpyDeviceToDevice, st));
    if (in.norm)
        OV_CUDA(c, cudaMemcpyAsync(out.norm, in.norm, norm_bytes(in.prec, in.nrhs, in.Vh), cudaMemcpyDeviceToDevice,
                                   st));
    return OV_OK;
}

// D(m) in, optionally followed by gamma5 (g5_out).  Sign by Eq. 7; the
// polynomial P(Q^2) psi_h by Clenshaw's recurrence in the variable
// Y = (2 Q^2 - (1+eps)) / (1-eps):
//   b_k = c_k psi_h + 2 Y b_{k+1} - b_{k+2},  k = n .. 1,   P psi_h = c_0 psi_h + Y b_1 - b_2,
// with 2 Y b = alpha H_w^2 b + beta b, alpha = 4 / (lmax^2 (1-eps)), beta = -2 (1+eps)/(1-eps).
// Each step is two dslash launches: t = H_w b_{k+1}, then H_w t with the
// whole combination fused into the epilogue.  b_n and b_{n-1} are kept as
// multiples of psi_h until a buffer is needed, so the launch count is 2n + 1.
// Finally D(m) psi = (rho + m/2) psi + (rho - m/2) [D_w(P psi_h) / lmax + gamma5 sum_i sign(lam_i) c_i eta_i]
// (gamma5 Q = D_w / lmax), in one more launch.
// gprec: precision of the links (-1: that of the fields); dots16: the low-mode coefficients may come
// from the bf16 tensor-core contraction (the operator's fields are 16-bit)
static int overlap_core(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, int g5_out,
                        cudaStream_t st, int poly, int gprec, bool dots16)
{
    // poly 1: the inner polynomial of the adaptive-precision CG (lower degree, same [eps, 1])
    const std::vector<double>& coef = poly ? c->coef_in : c->coef;
    const int degree = poly ? c->degree_in : c->degree;
    if (!c->have_gauge) return set_err(c, OV_ESTATE, "overlap: no gauge field (call ov_set_gauge)");
    if (!c->have_poly) return set_err(c, OV_ESTATE, "overlap: no sign polynomial (call ov_set_sign_poly)");
    const int P = in.prec, R = in.nrhs;
    const double rho = c->rho, lam = c->lmax, eps = c->eps;
    const double aw = 4.0 - rho;
    FieldDesc ph, w, t, B[3];
    OV_TRY(ws_field(c, WS_T, P, R, &t));
    OV_TRY(ws_field(c, WS_B0, P, R, &B[0]));
    OV_TRY(ws_field(c, WS_B1, P, R, &B[1]));
    OV_TRY(ws_field(c, WS_B2, P, R, &B[2]));
    const EigSet& E = c->eig[0];
    const bool defl = E.nev > 0;
    FieldDesc src = in;
    if (defl) {
        OV_TRY(ws_field(c, WS_PH, P, R, &ph));
        OV_TRY(ws_field(c, WS_W, P, R, &w));
        FieldDesc eta;
        OV_TRY(eig_vectors(c, 0, P, st, &eta));
        const int nblk = reduce_blocks(c->g);
        const int nparts = nblk * proj_groups(R);
        const size_t ncoef = (size_t)E.nev * R;
        OV_TRY(ensure_partials(c, nparts * ncoef * sizeof(double2)));
        if (ncoef * 2 > (size_t)DSCAL_COEF) return set_err(c, OV_EINVAL, "overlap: nev * nrhs = %zu too large", ncoef);
        double2* dcoef = (double2*)c->dscal;
        // tensor cores (tcgen05): c = eta^dag psi for 16-bit storage (bf16 operands), and the V c update
        // for FP32 (bf16 rows plus their bf16 remainders) and 16-bit storage; FP64 and double-float stay on
        // the CUDA cores
        const bool tc_ok = c->proj_tc && E.nev <= 128 && R <= 16 && c->g.Vh % 8 == 0;
        const bool tc = tc_ok && (P == P_F16 || P == P_BF16 || P == P_F32);
        (void)dots16;
        if (tc) {
            // FP32 work fields (also those of the 16-bit operator): bf16 rows plus their remainders
            OV_TRY(proj_dots_tc(c, 0, in, dcoef, st, P == P_F32 ? 2 : 1));
        } else {
            OV_CUDA(c, launch_proj_dots(c->g, eta, E.nev, in, (double2*)c->partials, nblk, st));
            OV_CUDA(c, launch_proj_finalize((double2*)c->partials, nparts, (int)ncoef, dcoef, st));
        }
        // the update of one FP32 right-hand side streams the rows once on the CUDA cores, faster than the
        // tensor cores' rows plus remainder rows (measured 0.24 against 0.32 ms at 16^3 x 32, 100 rows)
        if (tc && !(P == P_F32 && R == 1))
            OV_TRY(proj_update_tc(c, 0, in, dcoef, E.d_sign, ph, w, st));
        else
            OV_CUDA(c, launch_proj_update(c->g, eta, E.nev, dcoef, E.d_sign, in, ph, w, st));
        src = ph;
    }
    if (c->sign_backend == 1) {
        // Eq. 12: P(Q^2) psi_h = sum_i b_i (Q^2 + c_i)^-1 psi_h by multi-shift CG, then the same final launch
        OV_TRY(ws_field(c, WS_RS, P, R, &B[0]));
        OV_TRY(rational_solve(c, src, B[0], gprec, st));
        const double kk = (rho - 0.5 * mass) / lam;
        FieldDesc y[2] = {in, defl ? w : in};
        double sy[2] = {rho + 0.5 * mass, rho - 0.5 * mass};
        return dslash_apply(c, B[0], out, kk * aw, -0.5 * kk, 0, g5_out, defl ? 2 : 1, y, sy, st, gprec);
    }
    const double alpha = 4.0 / (lam * lam * (1.0 - eps));
    const double beta = -2.0 * (1.0 + eps) / (1.0 - eps);
    struct BRef {
        int buf;   // >= 0: value is B[buf]; -1: value is g * psi_h
        double g;
    };
    BRef b1{-1, 0.0}, b2{-1, 0.0};
    for (int k = degree; k >= 0; --k) {
        const double f = k == 0 ? 0.5 : 1.0;
        if (b1.buf < 0 && b1.g == 0.0) {  // b_{k+1} = 0 (then b_{k+2} = 0 too)
            BRef nb{-1, coef[k] - (b2.buf < 0 ? b2.g : 0.0)};
            b2 = b1;
            b1 = nb;
            continue;
        }
        FieldDesc y[3];
        double sy[3];
        int ny = 1;
        double psi_coef = coef[k];
        const FieldDesc* hin;
        double hscale;
        if (b1.buf < 0) {
            hin = &src;
            hscale = b1.g;
            psi_coef += f * beta * b1.g;
        } else {
            hin = &B[b1.buf];
            hscale = 1.0;
            y[ny] = B[b1.buf];
            sy[ny++] = f * beta;
        }
        int outbuf;
        if (b2.buf >= 0) {
            y[ny] = B[b2.buf];
            sy[ny++] = -1.0;
            outbuf = b2.buf;
        } else {
            psi_coef -= b2.g;
            outbuf = b1.buf == 0 ? 1 : 0;
        }
        y[0] = src;
        sy[0] = psi_coef;
        // t = H_w b_{k+1} (unscaled), then b_k = f alpha hscale H_w t + sum_j sy_j y_j
        OV_TRY(dslash_apply(c, *hin, t, aw, -0.5, 1, 0, 0, nullptr, nullptr, st, gprec));
        const double sc = f * alpha * hscale;
        OV_TRY(dslash_apply(c, t, B[outbuf], sc * aw, -0.5 * sc, 1, 0, ny, y, sy, st, gprec));
        b2 = b1;
        b1 = BRef{outbuf, 0.0};
    }
    // out = kk D_w(P) + (rho + m/2) in + (rho - m/2) W'
    const double kk = (rho - 0.5 * mass) / lam;
    const FieldDesc* pin = b1.buf >= 0 ? &B[b1.buf] : &src;
    const double psc = b1.buf >= 0 ? 1.0 : b1.g;
    FieldDesc y[2] = {in, defl ? w : in};
    double sy[2] = {rho + 0.5 * mass, rho - 0.5 * mass};
    OV_TRY(dslash_apply(c, *pin, out, kk * psc * aw, -0.5 * kk * psc, 0, g5_out, defl ? 2 : 1, y, sy, st, gprec));
    return OV_OK;
}

// D(m) in (gamma5 D(m) in if g5_out).  16-bit fields (option "clenshaw_f32", the default): the
// recurrence's work vectors are FP32 while the links stay 16-bit and the operator's input and output
// keep their 16-bit storage.  A Clenshaw sum of degree n carries the roundings of its n stored b_k
// through the remaining steps (the second-kind Chebyshev polynomials grow towards the ends of
// [eps, 1]), so 16-bit b_k put the overlap above 1e-3 where the lowest undeflated mode sits at the
// interval's edge; FP32 b_k leave the input, output and link roundings.  The kernel is bound by
// latency and issue, not bytes, so the FP32 work vectors cost little time.
static int overlap_apply_g5(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, int g5_out,
                            cudaStream_t st, int poly = 0)
{
    const int P = in.prec;
    if (!(c->clenshaw_f32 && (P == P_F16 || P == P_BF16))) return overlap_core(c, in, out, mass, g5_out, st, poly, -1, false);
    FieldDesc i32, o32;
    OV_TRY(ws_field(c, WS_MX0, P_F32, in.nrhs, &i32));
    OV_TRY(ws_field(c, WS_MX1, P_F32, in.nrhs, &o32));
    OV_TRY(convert(c, in, i32, st));
    OV_TRY(overlap_core(c, i32, o32, mass, g5_out, st, poly, P, true));
    return convert(c, o32, out, st);
}

void eig_clear(ov_ctx* c, EigSet& E)
{
    for (auto& f : E.vec) field_free(c, &f);
    if (E.d_sign) dev_free(c, E.d_sign, sizeof(double) * E.nev);
    if (E.tc_rows) dev_free(c, E.tc_rows, E.tc_bytes);
    if (E.tc_lo) dev_free(c, E.tc_lo, E.tc_lo_bytes);
    E.d_sign = nullptr;
    E.tc_rows = nullptr;
    E.tc_bytes = 0;
    E.tc_lo = nullptr;
    E.tc_lo_bytes = 0;
    E.nev = 0;
    E.vals.clear();
}

void graphs_clear(ov_ctx* c)
{
    if (c->graphs.empty()) return;
    cudaDeviceSynchronize();
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
    c->graphs.clear();
}

// Run `body(s)` (a fixed sequence of kernel launches on stream s) through a
// captured CUDA graph: the first call for a key runs eagerly (allocating any
// workspace) and then captures the same sequence; later calls replay it.  The
// legacy default stream (st == NULL) cannot be captured, so for it the graph
// runs on a library-owned non-blocking stream ordered after st by one event
// and followed by st through another: stream order is what the caller asked for.
template <typename F>
static int with_graph(ov_ctx* c, int kind, const FieldDesc& in, const FieldDesc& out, double mass, int g5,
                      cudaStream_t st, F body)
{
    // the rational sign is a host-driven iteration (convergence tests between launches): never captured
    if (!c->use_graphs || c->sign_backend == 1) return body(st);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st != nullptr && (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone))
        return body(st);  // the caller is capturing: record the launches into its graph
    cudaStream_t gs = st;
    if (st == nullptr) {
        if (!c->gstream) {
            OV_CUDA(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
            OV_CUDA(c, cudaEventCreateWithFlags(&c->gev[0], cudaEventDisableTiming));
            OV_CUDA(c, cudaEventCreateWithFlags(&c->gev[1], cudaEventDisableTiming));
        }
        gs = c->gstream;
        OV_CUDA(c, cudaEventRecord(c->gev[0], st));
        OV_CUDA(c, cudaStreamWaitEvent(gs, c->gev[0], 0));
    }
    auto join = [&]() -> int {
        if (gs != st) {
            OV_CUDA(c, cudaEventRecord(c->gev[1], gs));
            OV_CUDA(c, cudaStreamWaitEvent(st, c->gev[1], 0));
        }
        return OV_OK;
    };
    auto key = std::make_tuple(kind, (const void*)in.data, (const void*)out.data, in.prec, in.nrhs, mass, g5);
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
        OV_CUDA(c, cudaGraphLaunch(it->second.first, gs));
        c->dslash_launches += it->second.second;
        c->graph_replays++;
        return join();
    }
    {
        const int s0 = body(gs);
        if (s0 != OV_OK) {
            join();
            return s0;
        }
    }
    const long long before = c->dslash_launches;
    OV_CUDA(c, cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
    int s = body(gs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(gs, &g);
    const long long n = c->dslash_launches - before;
    c->dslash_launches = before;
    if (s != OV_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        join();
        return s != OV_OK ? s : set_err(c, OV_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        join();
        return set_err(c, OV_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    c->graphs[key] = {ex, n};
    c->graph_captures++;
    return join();
}

int overlap_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, cudaStream_t st)
{
    return with_graph(c, 0, in, out, mass, 0, st,
                      [&](cudaStream_t s) { return overlap_apply_g5(c, in, out, mass, 0, s); });
}

int overlap_g5_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, int g5_out, cudaStream_t st)
{
    return with_graph(c, 3, in, out, mass, g5_out, st,
                      [&](cudaStream_t s) { return overlap_apply_g5(c, in, out, mass, g5_out, s); });
}

int normal_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, cudaStream_t st, int poly)
{
    FieldDesc u;
    OV_TRY(ws_field(c, WS_AUX0, in.prec, in.nrhs, &u));
    return with_graph(c, 1 + 16 * poly, in, out, mass, 0, st, [&](cudaStream_t s) {
        OV_TRY(overlap_apply_g5(c, in, u, mass, 1, s, poly));  // u = g5 D in
        return overlap_apply_g5(c, u, out, mass, 1, s, poly);  // out = g5 D g5 D in = D^dag D in
    });
}

// D(m)^dag D(m) on one chiral sector (Sec. V: chiral basis, sources and
// eigenvectors of definite chirality).  With sign^2 = 1 and gamma5 psi = chi psi,
//   P D(m)^dag D(m) P psi = m^2 psi + (rho^2 - m^2/4)/rho (1 + chi gamma5) D(0) psi,
// P = (1 + chi gamma5)/2: one sign application instead of two (exact up to the
// polynomial's error delta).  dcoef: device double2 [3][R] =
// (m^2, (rho^2 - m^2/4)/rho, chi_r (rho^2 - m^2/4)/rho), per right-hand side.
int chiral_apply(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double mass, const double2* dcoef,
                 cudaStream_t st, int poly)
{
    FieldDesc u;
    OV_TRY(ws_field(c, WS_AUX0, in.prec, in.nrhs, &u));
    return with_graph(c, 2 + 16 * poly, in, out, mass, 0, st, [&](cudaStream_t s) {
        OV_TRY(overlap_apply_g5(c, in, u, 0.0, 0, s, poly));  // u = D(0) in
        FieldDesc v[3] = {in, u, u};
        return lincomb(c, out, 3, v, nullptr, dcoef, 4, nullptr, s);
    });
}

// Chirality chi_r of every right-hand side of f (f^dag gamma5 f = chi |f|^2 to 1e-12, else
// OV_EINVAL) and the chiral-sector coefficients at DSCAL_CHCO: [3][R] for chiral_apply, then
// [2][R] = (1/2, chi/2) for the sector projection.  tmp: a field of f's shape (overwritten).
int chiral_setup(ov_ctx* c, const FieldDesc& f, const FieldDesc& tmp, double mass, cudaStream_t st)
{
    const int R = f.nrhs;
    if (5 * R * 2 > DSCAL_NORM - DSCAL_CHCO) return set_err(c, OV_EINVAL, "chiral: too many right-hand sides");
    double2* ddt = (double2*)(c->dscal + DSCAL_DOT);
    std::vector<double2> hn(R), hg(R);
    OV_TRY(norm2(c, f, (double*)ddt, st));
    OV_CUDA(c, cudaMemcpyAsync(hn.data(), ddt, R * sizeof(double2), cudaMemcpyDeviceToHost, st));
    FieldDesc v1[1] = {f};
    const double2 one[1] = {make_double2(1, 0)};
    OV_TRY(lincomb(c, tmp, 1, v1, one, nullptr, 1, nullptr, st));  // tmp = gamma5 f
    OV_TRY(dot(c, f, tmp, ddt, st));
    OV_CUDA(c, cudaMemcpyAsync(hg.data(), ddt, R * sizeof(double2), cudaMemcpyDeviceToHost, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    const double cm = (c->rho * c->rho - 0.25 * mass * mass) / c->rho;
    std::vector<double2> hc(5 * R);
    for (int q = 0; q < R; ++q) {
        const double n2 = hn[q].x;  // a zero right-hand side lies in both sectors
        if (!(n2 >= 0) || !(std::fabs(std::fabs(hg[q].x) - n2) <= 1e-12 * n2))
            return set_err(c, OV_EINVAL, "chiral mode needs right-hand sides of definite chirality (rhs %d)", q);
        const double chi = hg[q].x >= 0 ? 1.0 : -1.0;
        hc[q] = make_double2(mass * mass, 0);
        hc[R + q] = make_double2(cm, 0);
        hc[2 * R + q] = make_double2(chi * cm, 0);
        hc[3 * R + q] = make_double2(0.5, 0);
        hc[4 * R + q] = make_double2(0.5 * chi, 0);
    }
    OV_CUDA(c, cudaMemcpyAsync(c->dscal + DSCAL_CHCO, hc.data(), hc.size() * sizeof(double2),
                               cudaMemcpyHostToDevice, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    return OV_OK;
}

// Chebyshev-interpolant coefficients of x^{-1/2} on [eps, 1] at the n+1
// Chebyshev nodes of the variable y = (2x - (1+eps))/(1-eps) (Eq. 4, Sec. V);
// c_0 is halved so that P = sum_k c_k T_k(y).
static void cheb_coefficients(double eps, int n, std::vector<double>& c)
{
    const int m = n + 1;
    std::vector<double> f(m);
    for (int j = 0; j < m; ++j) {
        double th = M_PI * (j + 0.5) / m;
        f[j] = 1.0 / std::sqrt(0.5 * (1.0 + eps) + 0.5 * (1.0 - eps) * std::cos(th));
    }
    c.assign(m, 0.0);
    for (int k = 0; k < m; ++k) {
        double s = 0;
        for (int j = 0; j < m; ++j) s += f[j] * std::cos(M_PI * k * (j + 0.5) / m);
        c[k] = 2.0 * s / m;
    }
    c[0] *= 0.5;
}

// delta = max over [eps, 1] of |1 - sqrt(x) P(x)| (Eq. 4) for the interpolant c, on a grid of points
// uniform in sqrt(x) (the error oscillates fastest near eps) plus the end points
static double poly_delta(const std::vector<double>& cf, double eps)
{
    const int n = (int)cf.size() - 1;
    const int npts = 4000;
    double worst = 0.0;
    for (int i = 0; i <= npts; ++i) {
        const double sx = std::sqrt(eps) + (1.0 - std::sqrt(eps)) * i / npts;
        const double x = sx * sx;
        const double y = (2.0 * x - (1.0 + eps)) / (1.0 - eps);
        double b1 = 0, b2 = 0;  // Clenshaw for sum_k c_k T_k(y)
        for (int k = n; k >= 1; --k) {
            const double b0 = cf[k] + 2.0 * y * b1 - b2;
            b2 = b1;
            b1 = b0;
        }
        const double P = cf[0] + y * b1 - b2;
        worst = std::max(worst, std::fabs(1.0 - sx * P));
    }
    return worst;
}

// Inner polynomial of the adaptive-precision CG: the lowest degree (<= the accurate one) whose delta on
// [eps, 1] is at most c->adaptive_delta; off (degree_in = degree) when adaptive_delta is 0.
static void set_inner_poly(ov_ctx* c)
{
    c->degree_in = c->degree;
    c->coef_in = c->coef;
    if (!(c->adaptive_delta > 0)) return;
    std::vector<double> cf;
    for (int n = 1; n < c->degree; ++n) {
        cheb_coefficients(c->eps, n, cf);
        if (poly_delta(cf, c->eps) <= c->adaptive_delta) {
            c->degree_in = n;
            c->coef_in = cf;
            return;
        }
    }
}

// ---- rational sign (Eq. 12): Zolotarev's optimal partial fractions of x^{-1/2} on [eps, 1] ----
// K(m) and the Jacobi functions of parameter m by the arithmetic-geometric mean (Gauss; Abramowitz and
// Stegun 17.6 and 16.4): the AGM sequence a_j, b_j, c_j = (a_{j-1} - b_{j-1})/2 from (1, sqrt(1-m), sqrt m),
// K = pi / (2 a_N); am(u) from phi_N = 2^N a_N u by phi_{j-1} = (phi_j + asin(c_j sin phi_j / a_j)) / 2.
static void agm_jacobi(double u, double m, double* sn, double* cn, double* K)
{
    std::vector<double> av{1.0}, cv{std::sqrt(m)};
    double bb = std::sqrt(1.0 - m);
    while (av.size() < 64 && std::fabs(cv.back()) > 1e-17) {
        const double a0 = av.back();
        av.push_back(0.5 * (a0 + bb));
        cv.push_back(0.5 * (a0 - bb));
        bb = std::sqrt(a0 * bb);
    }
    const int N = (int)av.size() - 1;
    if (K) *K = M_PI / (2.0 * av[N]);
    double phi = std::ldexp(av[N] * u, N);
    for (int j = N; j >= 1; --j) phi = 0.5 * (phi + std::asin(cv[j] * std::sin(phi) / av[j]));
    *sn = std::sin(phi);
    *cn = std::cos(phi);
}

// sign(q) ~ D q prod_{j<n} (q^2 + z_j) / prod_{i<=n} (q^2 + p_i) on sqrt(eps) <= |q| <= 1 with
// z_j = a_{2j}, p_i = a_{2i-1}, a_l = eps sn^2 / cn^2 (l K'/(2n) | 1 - eps), K' = K(1 - eps) (Zolotarev);
// D makes the error equioscillate (2 / (max + min) of the unscaled function on [sqrt(eps), 1], its extremes
// bracketed on a log grid and refined by golden section).  Output: P(x) = sum_i b_i / (x + c_i), delta.
static double zolotarev_fractions(double eps, int n, std::vector<double>& b, std::vector<double>& cc)
{
    std::vector<double> a(2 * n + 1, 0.0);
    double Kp = 0, sn = 0, cn = 0;
    agm_jacobi(0.0, 1.0 - eps, &sn, &cn, &Kp);
    for (int l = 1; l <= 2 * n - 1; ++l) {
        agm_jacobi(l * Kp / (2.0 * n), 1.0 - eps, &sn, &cn, nullptr);
        a[l] = eps * (sn * sn) / (cn * cn);
    }
    auto f = [&](double q) {
        double v = q;
        for (int j = 1; j < n; ++j) v *= q * q + a[2 * j];
        for (int i = 1; i <= n; ++i) v /= q * q + a[2 * i - 1];
        return v;
    };
    auto refine = [&](double lo, double hi, bool top) {
        const double g = 0.6180339887498949;
        for (int it = 0; it < 160; ++it) {
            const double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
            if ((f(x1) > f(x2)) == top)
                hi = x2;
            else
                lo = x1;
        }
        return f(0.5 * (lo + hi));
    };
    const double k = std::sqrt(eps);
    double hi = std::max(f(k), f(1.0)), lo = std::min(f(k), f(1.0));
    const int G = 12000;
    std::vector<double> q(G + 1), v(G + 1);
    for (int i = 0; i <= G; ++i) {
        q[i] = k * std::pow(1.0 / k, (double)i / G);
        v[i] = f(q[i]);
    }
    for (int i = 1; i < G; ++i) {
        if (v[i] > v[i - 1] && v[i] >= v[i + 1]) hi = std::max(hi, refine(q[i - 1], q[i + 1], true));
        if (v[i] < v[i - 1] && v[i] <= v[i + 1]) lo = std::min(lo, refine(q[i - 1], q[i + 1], false));
    }
    const double D = 2.0 / (hi + lo);
    b.assign(n, 0.0);
    cc.assign(n, 0.0);
    for (int i = 1; i <= n; ++i) {
        const double ci = a[2 * i - 1];
        double w = D;
        for (int j = 1; j < n; ++j) w *= a[2 * j] - ci;
        for (int l = 1; l <= n; ++l)
            if (l != i) w /= a[2 * l - 1] - ci;
        cc[i - 1] = ci;
        b[i - 1] = w;
    }
    return (hi - lo) / (hi + lo);
}

static int check_prec(ov_ctx* c, int prec)
{
    if (prec < 0 || prec >= NPREC) return set_err(c, OV_EINVAL, "unknown precision %d", prec);
    return OV_OK;
}

}  // namespace ov

// ===========================================================================
// exported C ABI
// ===========================================================================
extern "C" {

int ov_create(ov_ctx** ctx, const int dims[4], const double bc_phase[4])
{
    if (!ctx || !dims || !bc_phase) return OV_EINVAL;
    *ctx = nullptr;
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] < 2 || dims[mu] % 2) return OV_EINVAL;
    long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V / 2 > (1LL << 26)) return OV_EINVAL;  // keeps every 16-byte chunk index below 2^31
    ov_ctx* c = new ov_ctx();
    for (int mu = 0; mu < 4; ++mu) {
        c->dims[mu] = dims[mu];
        c->bc[mu] = bc_phase[mu];
        c->g.L[mu] = dims[mu];
        c->g.bc[mu] = bc_phase[mu];
        c->g.fbc[mu] = (float)bc_phase[mu];
    }
    c->g.Lxh = dims[0] / 2;
    c->g.Vh = (int)(V / 2);
    c->g.fxh = FastDiv((uint32_t)c->g.Lxh);
    c->g.fy = FastDiv((uint32_t)dims[1]);
    c->g.fz = FastDiv((uint32_t)dims[2]);
    cudaGetDevice(&c->device);
    void* p = nullptr;
    if (dev_alloc(c, &p, DSCAL_DOUBLES * sizeof(double)) != OV_OK) {
        delete c;
        return OV_ENOMEM;
    }
    c->dscal = (double*)p;
    if (dev_alloc(c, &p, 64) != OV_OK) {
        dev_free(c, c->dscal, DSCAL_DOUBLES * sizeof(double));
        delete c;
        return OV_ENOMEM;
    }
    c->derr = (unsigned*)p;
    if (cudaMemset(c->derr, 0, 64) != cudaSuccess) {
        ov_destroy(c);
        return OV_ECUDA;
    }
    *ctx = c;
    return OV_OK;
}

int ov_destroy(ov_ctx* c)
{
    if (!c) return OV_EINVAL;
    cudaDeviceSynchronize();
    graphs_clear(c);
    net_free(c);
    for (int p = 0; p < NPREC; ++p)
        if (c->gauge[p]) dev_free(c, c->gauge[p], (size_t)8 * c->g.Vh * gauge_link_bytes(p));
    for (auto& e : c->eig) eig_clear(c, e);
    for (auto& kv : c->ws) field_free(c, &kv.second);
    if (c->partials) dev_free(c, c->partials, c->partials_bytes);
    if (c->tc_b) dev_free(c, c->tc_b, c->tc_b_bytes);
    if (c->tc_cb) dev_free(c, c->tc_cb, c->tc_cb_bytes);
    if (c->rcoef) dev_free(c, c->rcoef, c->rcoef_bytes);
    if (c->tc_err) dev_free(c, c->tc_err, sizeof(int));
    for (int i = 0; i < 2; ++i)
        if (c->stage[i]) dev_free(c, c->stage[i], c->stage_bytes[i]);
    dev_free(c, c->dscal, DSCAL_DOUBLES * sizeof(double));
    dev_free(c, c->derr, 64);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    for (auto& e : c->gev)
        if (e) cudaEventDestroy(e);
    delete c;
    return OV_OK;
}

const char* ov_last_error(const ov_ctx* c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

int ov_set_gauge(ov_ctx* c, const void* U, void* stream)
{
    if (!c || !U) return c ? set_err(c, OV_EINVAL, "set_gauge: null pointer") : OV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)2 * c->g.Vh * 4 * 9 * 16;
    const double* dU = nullptr;
    OV_TRY(stage_in(c, 0, U, bytes, st, &dU));
    for (int p = 0; p < NPREC; ++p) {
        if (!c->gauge[p]) OV_TRY(dev_alloc(c, &c->gauge[p], (size_t)8 * c->g.Vh * gauge_link_bytes(p)));
    }
    OV_CUDA(c, cudaMemsetAsync(c->derr, 0, 2 * sizeof(unsigned), st));
    for (int p = 0; p < NPREC; ++p) OV_CUDA(c, launch_pack_gauge(c->g, dU, c->gauge[p], p, p == 0 ? c->derr : nullptr, st));
    unsigned herr[2];
    OV_CUDA(c, cudaMemcpyAsync(herr, c->derr, sizeof herr, cudaMemcpyDeviceToHost, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    float e_unit, e_row;
    memcpy(&e_unit, &herr[0], 4);
    memcpy(&e_row, &herr[1], 4);
    if (!(e_unit <= 1e-9f) || !(e_row <= 1e-9f)) {
        c->have_gauge = false;
        return set_err(c, OV_EINVAL,
                       "set_gauge: links are not SU(3) (max |U U^dag - 1| = %g, max |row2 - conj(row0 x row1)| = %g); "
                       "reconstruct-12 needs SU(3)",
                       (double)e_unit, (double)e_row);
    }
    c->have_gauge = true;
    graphs_clear(c);
    // eigenpairs of a previous gauge field no longer apply
    for (auto& e : c->eig) eig_clear(c, e);
    return OV_OK;
}

static int apply_canonical(ov_ctx* c, const void* in, void* out, double m, int nrhs, int prec, void* stream, int kind)
{
    if (!c) return OV_EINVAL;
    if (!in || !out) return set_err(c, OV_EINVAL, "null buffer");
    if (in == out) return set_err(c, OV_EINVAL, "in and out must differ");
    OV_TRY(check_prec(c, prec));
    if (nrhs < 1 || nrhs > 16) return set_err(c, OV_EINVAL, "nrhs = %d out of range 1..16", nrhs);
    if (!c->have_gauge) return set_err(c, OV_ESTATE, "no gauge field (call ov_set_gauge)");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)nrhs * 2 * c->g.Vh * 12 * 16;
    const double* din = nullptr;
    double* dout = nullptr;
    OV_TRY(stage_in(c, 0, in, bytes, st, &din));
    OV_TRY(stage_out_buffer(c, 1, out, bytes, &dout));
    FieldDesc fi, fo;
    OV_TRY(ws_field(c, WS_IN, prec, nrhs, &fi));
    OV_TRY(ws_field(c, WS_OUT, prec, nrhs, &fo));
    OV_CUDA(c, launch_pack(c->g, din, fi, 0, st));
    if (kind == 2) {
        OV_TRY(overlap_apply(c, fi, fo, m, st));
    } else if (kind == 3) {
        OV_TRY(normal_apply(c, fi, fo, m, st));
    } else if (kind == 4) {
        OV_TRY(chiral_setup(c, fi, fo, m, st));
        OV_TRY(chiral_apply(c, fi, fo, m, (const double2*)(c->dscal + DSCAL_CHCO), st));
    } else {
        OV_TRY(dslash_apply(c, fi, fo, 4.0 + m, -0.5, kind == 1, 0, 0, nullptr, nullptr, st));
    }
    OV_CUDA(c, launch_unpack(c->g, fo, dout, 0, st));
    OV_TRY(stage_out_finish(c, out, dout, bytes, st));
    return check_kernel_flags(c, st);
}

int ov_apply_dslash(ov_ctx* c, const void* in, void* out, double m, int nrhs, int prec, void* stream)
{
    return apply_canonical(c, in, out, m, nrhs, prec, stream, 0);
}

int ov_apply_Hw(ov_ctx* c, const void* in, void* out, double m, int nrhs, int prec, void* stream)
{
    return apply_canonical(c, in, out, m, nrhs, prec, stream, 1);
}

int ov_apply_overlap(ov_ctx* c, const void* in, void* out, double mass, int nrhs, int prec, void* stream)
{
    if (!c) return OV_EINVAL;
    if (!c->have_poly) return set_err(c, OV_ESTATE, "overlap: no sign polynomial (call ov_set_sign_poly)");
    return apply_canonical(c, in, out, mass, nrhs, prec, stream, 2);
}

int ov_apply_normal(ov_ctx* c, const void* in, void* out, double mass, int nrhs, int prec, int chiral,
                    void* stream)
{
    if (!c) return OV_EINVAL;
    if (!c->have_poly) return set_err(c, OV_ESTATE, "normal: no sign polynomial (call ov_set_sign_poly)");
    return apply_canonical(c, in, out, mass, nrhs, prec, stream, chiral ? 4 : 3);
}

int ov_set_sign_poly(ov_ctx* c, double rho, double eps, int degree, double lambda_max)
{
    if (!c) return OV_EINVAL;
    if (!(eps > 0.0 && eps < 1.0)) return set_err(c, OV_EINVAL, "eps = %g outside (0, 1)", eps);
    if (degree < 0 || degree > 100000) return set_err(c, OV_EINVAL, "degree = %d out of range", degree);
    if (!(rho > 0.0 && rho < 2.0)) return set_err(c, OV_EINVAL, "rho = %g outside (0, 2)", rho);
    graphs_clear(c);
    c->rho = rho;
    c->eps = eps;
    c->degree = degree;
    c->sign_backend = 0;
    cheb_coefficients(eps, degree, c->coef);
    set_inner_poly(c);
    if (lambda_max > 0) {
        c->lmax = lambda_max;
    } else {
        if (!c->have_gauge) return set_err(c, OV_ESTATE, "lambda_max estimate needs the gauge field");
        double l = 0;
        OV_TRY(estimate_lambda_max(c, 50, &l, (cudaStream_t)0));
        c->lmax = 1.01 * l;
    }
    c->have_poly = true;
    return OV_OK;
}

int ov_set_sign_rational(ov_ctx* c, double rho, double eps, int npoles, double lambda_max)
{
    if (!c) return OV_EINVAL;
    if (!(eps > 0.0 && eps < 1.0)) return set_err(c, OV_EINVAL, "eps = %g outside (0, 1)", eps);
    if (npoles < 1 || npoles > 64) return set_err(c, OV_EINVAL, "npoles = %d out of range 1..64", npoles);
    if (!(rho > 0.0 && rho < 2.0)) return set_err(c, OV_EINVAL, "rho = %g outside (0, 2)", rho);
    double l = lambda_max;
    if (!(l > 0)) {
        if (!c->have_gauge) return set_err(c, OV_ESTATE, "lambda_max estimate needs the gauge field");
        OV_TRY(estimate_lambda_max(c, 50, &l, (cudaStream_t)0));
        l *= 1.01;
    }
    graphs_clear(c);
    c->rho = rho;
    c->eps = eps;
    c->lmax = l;
    c->rdelta = zolotarev_fractions(eps, npoles, c->rb, c->rc);
    c->sign_backend = 1;
    c->have_poly = true;
    return OV_OK;
}

int ov_get_sign_rational(const ov_ctx* c, int* npoles, double* b, double* cc, double* delta)
{
    if (!c || !npoles) return OV_EINVAL;
    if (c->sign_backend != 1) return OV_ESTATE;
    *npoles = (int)c->rb.size();
    for (size_t i = 0; i < c->rb.size(); ++i) {
        if (b) b[i] = c->rb[i];
        if (cc) cc[i] = c->rc[i];
    }
    if (delta) *delta = c->rdelta;
    return OV_OK;
}

int ov_get_sign_poly(const ov_ctx* c, double* rho, double* eps, int* degree, double* lambda_max)
{
    if (!c) return OV_EINVAL;
    if (rho) *rho = c->rho;
    if (eps) *eps = c->eps;
    if (degree) *degree = c->degree;
    if (lambda_max) *lambda_max = c->lmax;
    return c->have_poly ? OV_OK : OV_ESTATE;
}

int ov_set_eigenpairs(ov_ctx* c, int which, int nev, const double* vals, const void* vecs, void* stream)
{
    if (!c) return OV_EINVAL;
    if (which != 0 && which != 1) return set_err(c, OV_EINVAL, "which = %d (0 or 1)", which);
    if (nev < 0 || nev > 2048) return set_err(c, OV_EINVAL, "nev = %d out of range 0..2048", nev);
    if (nev > 0 && (!vals || !vecs)) return set_err(c, OV_EINVAL, "null eigenpair buffers");
    cudaStream_t st = (cudaStream_t)stream;
    EigSet& E = c->eig[which];
    OV_CUDA(c, cudaStreamSynchronize(st));
    graphs_clear(c);
    eig_clear(c, E);
    if (nev == 0) return OV_OK;
    OV_TRY(field_alloc(c, P_F64, nev, &E.vec[P_F64]));
    const size_t one = (size_t)2 * c->g.Vh * 12 * 16;
    // pack in chunks of 16 vectors through the staging buffer
    for (int i0 = 0; i0 < nev; i0 += 16) {
        int n = nev - i0 < 16 ? nev - i0 : 16;
        const double* src = nullptr;
        OV_TRY(stage_in(c, 0, (const char*)vecs + one * i0, one * n, st, &src));
        FieldDesc sub = E.vec[P_F64];
        sub.nrhs = n;
        sub.data = E.vec[P_F64].data + (size_t)i0 * E.vec[P_F64].rhs_bytes();
        OV_CUDA(c, launch_pack(c->g, src, sub, 0, st));
        OV_CUDA(c, cudaStreamSynchronize(st));
    }
    E.nev = nev;
    E.vals.assign(vals, vals + nev);
    std::vector<double> sg(nev);
    for (int i = 0; i < nev; ++i) sg[i] = vals[i] > 0 ? 1.0 : (vals[i] < 0 ? -1.0 : 0.0);
    void* p = nullptr;
    OV_TRY(dev_alloc(c, &p, sizeof(double) * nev));
    E.d_sign = (double*)p;
    OV_CUDA(c, cudaMemcpy(E.d_sign, sg.data(), sizeof(double) * nev, cudaMemcpyHostToDevice));
    return OV_OK;
}

int ov_get_eigenpairs(ov_ctx* c, int which, int* nev, double* vals, void* vecs, void* stream)
{
    if (!c || !nev) return c ? set_err(c, OV_EINVAL, "null nev") : OV_EINVAL;
    if (which != 0 && which != 1) return set_err(c, OV_EINVAL, "which = %d (0 or 1)", which);
    cudaStream_t st = (cudaStream_t)stream;
    EigSet& E = c->eig[which];
    *nev = E.nev;
    if (vals)
        for (int i = 0; i < E.nev; ++i) vals[i] = E.vals[i];
    if (vecs && E.nev) {
        const size_t one = (size_t)2 * c->g.Vh * 12 * 16;
        for (int i0 = 0; i0 < E.nev; i0 += 16) {
            int n = E.nev - i0 < 16 ? E.nev - i0 : 16;
            double* dst = nullptr;
            void* hdst = (char*)vecs + one * i0;
            OV_TRY(stage_out_buffer(c, 1, hdst, one * n, &dst));
            FieldDesc sub = E.vec[P_F64];
            sub.nrhs = n;
            sub.data = E.vec[P_F64].data + (size_t)i0 * E.vec[P_F64].rhs_bytes();
            OV_CUDA(c, launch_unpack(c->g, sub, dst, 0, st));
            OV_TRY(stage_out_finish(c, hdst, dst, one * n, st));
        }
        OV_CUDA(c, cudaStreamSynchronize(st));
    }
    return OV_OK;
}

int ov_deflate(ov_ctx* c, int which, int nev, double tol, void* stream)
{
    if (!c) return OV_EINVAL;
    if (which != 0 && which != 1) return set_err(c, OV_EINVAL, "which = %d (0 or 1)", which);
    if (nev < 1 || nev > 1024) return set_err(c, OV_EINVAL, "nev = %d out of range 1..1024", nev);
    if (!(tol > 0)) return set_err(c, OV_EINVAL, "tol must be positive");
    if (!c->have_gauge) return set_err(c, OV_ESTATE, "deflate: no gauge field");
    if (which == 1 && !c->have_poly) return set_err(c, OV_ESTATE, "deflate(which=1): no sign polynomial");
    return deflate_impl(c, which, nev, tol, (cudaStream_t)stream);
}

int ov_cg_solve(ov_ctx* c, const void* b, void* x, int nrhs, double mass, double tol, int max_iter, int precond,
                int inner_prec, ov_solve_info* info, void* stream)
{
    if (!c) return OV_EINVAL;
    if (!b || !x) return set_err(c, OV_EINVAL, "null buffer");
    if (b == x) return set_err(c, OV_EINVAL, "b and x must differ");
    if (nrhs < 1 || nrhs > 16) return set_err(c, OV_EINVAL, "nrhs = %d out of range 1..16", nrhs);
    if (!(tol > 0) || max_iter < 1) return set_err(c, OV_EINVAL, "tol and max_iter must be positive");
    OV_TRY(check_prec(c, inner_prec));
    if (!c->have_gauge || !c->have_poly) return set_err(c, OV_ESTATE, "cg: needs gauge field and sign polynomial");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)nrhs * 2 * c->g.Vh * 12 * 16;
    const double* db = nullptr;
    double* dx = nullptr;
    OV_TRY(stage_in(c, 0, b, bytes, st, &db));
    OV_TRY(stage_out_buffer(c, 1, x, bytes, &dx));
    FieldDesc fb, fx;
    OV_TRY(ws_field(c, WS_CG_B, P_F64, nrhs, &fb));
    OV_TRY(ws_field(c, WS_CG_X, P_F64, nrhs, &fx));
    OV_CUDA(c, launch_pack(c->g, db, fb, 0, st));
    int s = cg_impl(c, fb, fx, mass, tol, max_iter, precond, inner_prec, info, st);
    if (s != OV_OK && s != OV_ENOTCONV && s != OV_ESTALL) return s;
    OV_CUDA(c, launch_unpack(c->g, fx, dx, 0, st));
    OV_TRY(stage_out_finish(c, x, dx, bytes, st));
    return s;
}

int ov_cg_solve_multimass(ov_ctx* c, const void* b, void* x, int nrhs, int nmass, const double* masses, double tol,
                          int max_iter, int inner_prec, int output, ov_solve_info* info, void* stream)
{
    if (!c) return OV_EINVAL;
    if (!b || !x || !masses) return set_err(c, OV_EINVAL, "null buffer");
    if (nrhs < 1 || nrhs > 16) return set_err(c, OV_EINVAL, "nrhs = %d out of range 1..16", nrhs);
    if (nmass < 1 || nmass > 16) return set_err(c, OV_EINVAL, "nmass = %d out of range 1..16", nmass);
    if (!(tol > 0) || max_iter < 1) return set_err(c, OV_EINVAL, "tol and max_iter must be positive");
    if (output < 0 || output > 2) return set_err(c, OV_EINVAL, "output = %d (0, 1 or 2)", output);
    for (int k = 0; k < nmass; ++k)
        if (!(masses[k] >= 0 && masses[k] < 2 * c->rho)) return set_err(c, OV_EINVAL, "mass %g outside [0, 2 rho)", masses[k]);
    OV_TRY(check_prec(c, inner_prec));
    if (!c->have_gauge || !c->have_poly) return set_err(c, OV_ESTATE, "multimass: needs gauge field and sign polynomial");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t one = (size_t)nrhs * 2 * c->g.Vh * 12 * 16;
    const double* db = nullptr;
    OV_TRY(stage_in(c, 0, b, one, st, &db));
    FieldDesc fb;
    OV_TRY(ws_field(c, WS_CG_B, P_F64, nrhs, &fb));
    OV_CUDA(c, launch_pack(c->g, db, fb, 0, st));
    // one accurate-precision solution field per mass (device memory for the duration of the call)
    std::vector<FieldDesc> fx(nmass);
    int s = OV_OK;
    for (int k = 0; k < nmass && s == OV_OK; ++k) s = field_alloc(c, c->hi_prec, nrhs, &fx[k]);
    if (s == OV_OK) s = multimass_impl(c, fb, fx.data(), nmass, masses, tol, max_iter, inner_prec, output, info, st);
    if (s == OV_OK || s == OV_ENOTCONV) {
        FieldDesc f64;
        int s2 = ws_field(c, WS_CG_X, P_F64, nrhs, &f64);
        for (int k = 0; k < nmass && s2 == OV_OK; ++k) {
            double* dx = nullptr;
            void* hx = (char*)x + one * k;
            s2 = stage_out_buffer(c, 1, hx, one, &dx);
            if (s2 == OV_OK) s2 = convert(c, fx[k], f64, st);
            if (s2 == OV_OK && launch_unpack(c->g, f64, dx, 0, st) != cudaSuccess)
                s2 = set_err(c, OV_ECUDA, "multimass: unpack failed");
            if (s2 == OV_OK) s2 = stage_out_finish(c, hx, dx, one, st);
        }
        if (s2 != OV_OK) s = s2;
    }
    cudaStreamSynchronize(st);
    for (auto& f : fx) field_free(c, &f);
    return s;
}

int ov_field_create(ov_ctx* c, int nrhs, int prec, ov_field** f)
{
    if (!c || !f) return c ? set_err(c, OV_EINVAL, "null pointer") : OV_EINVAL;
    OV_TRY(check_prec(c, prec));
    if (nrhs < 1 || nrhs > 16) return set_err(c, OV_EINVAL, "nrhs = %d out of range 1..16", nrhs);
    ov_field* h = new ov_field();
    h->owner = c;
    int s = field_alloc(c, prec, nrhs, &h->d);
    if (s != OV_OK) {
        delete h;
        return s;
    }
    *f = h;
    return OV_OK;
}

int ov_field_destroy(ov_field* f)
{
    if (!f) return OV_EINVAL;
    cudaDeviceSynchronize();
    field_free(f->owner, &f->d);
    delete f;
    return OV_OK;
}

int ov_field_import(ov_ctx* c, ov_field* f, const void* canonical, void* stream)
{
    if (!c || !f || !canonical) return c ? set_err(c, OV_EINVAL, "null pointer") : OV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)f->d.nrhs * 2 * c->g.Vh * 12 * 16;
    const double* src = nullptr;
    OV_TRY(stage_in(c, 0, canonical, bytes, st, &src));
    OV_CUDA(c, launch_pack(c->g, src, f->d, 0, st));
    return OV_OK;
}

int ov_field_export(ov_ctx* c, const ov_field* f, void* canonical, void* stream)
{
    if (!c || !f || !canonical) return c ? set_err(c, OV_EINVAL, "null pointer") : OV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)f->d.nrhs * 2 * c->g.Vh * 12 * 16;
    double* dst = nullptr;
    OV_TRY(stage_out_buffer(c, 1, canonical, bytes, &dst));
    OV_CUDA(c, launch_unpack(c->g, f->d, dst, 0, st));
    return stage_out_finish(c, canonical, dst, bytes, st);
}

int ov_dslash_field(ov_ctx* c, const ov_field* in, ov_field* out, double m, int gamma5, void* stream)
{
    if (!c || !in || !out) return c ? set_err(c, OV_EINVAL, "null pointer") : OV_EINVAL;
    if (in == out) return set_err(c, OV_EINVAL, "in and out must differ");
    if (in->d.prec != out->d.prec || in->d.nrhs != out->d.nrhs)
        return set_err(c, OV_EINVAL, "fields differ in precision or nrhs");
    if (!c->have_gauge) return set_err(c, OV_ESTATE, "no gauge field");
    return dslash_apply(c, in->d, out->d, 4.0 + m, -0.5, gamma5 ? 1 : 0, 0, 0, nullptr, nullptr,
                        (cudaStream_t)stream);
}

int ov_overlap_field(ov_ctx* c, const ov_field* in, ov_field* out, double mass, void* stream)
{
    if (!c || !in || !out) return c ? set_err(c, OV_EINVAL, "null pointer") : OV_EINVAL;
    if (in == out) return set_err(c, OV_EINVAL, "in and out must differ");
    if (in->d.prec != out->d.prec || in->d.nrhs != out->d.nrhs)
        return set_err(c, OV_EINVAL, "fields differ in precision or nrhs");
    return overlap_apply(c, in->d, out->d, mass, (cudaStream_t)stream);
}

int ov_field_dot(ov_ctx* c, const ov_field* x, const ov_field* y, double* out, void* stream)
{
    if (!c || !x || !y || !out) return c ? set_err(c, OV_EINVAL, "null pointer") : OV_EINVAL;
    if (x->d.prec != y->d.prec || x->d.nrhs != y->d.nrhs)
        return set_err(c, OV_EINVAL, "fields differ in precision or nrhs");
    cudaStream_t st = (cudaStream_t)stream;
    double* dev = nullptr;
    if (is_device_ptr(out)) {
        dev = out;
    } else {
        if (x->d.nrhs * 2 > 1024) return set_err(c, OV_EINVAL, "too many right-hand sides");
        dev = c->dscal + DSCAL_DOT;
    }
    OV_TRY(dot(c, x->d, y->d, (double2*)dev, st));
    if (dev != out) {
        OV_CUDA(c, cudaMemcpyAsync(out, dev, sizeof(double) * 2 * x->d.nrhs, cudaMemcpyDeviceToHost, st));
        OV_CUDA(c, cudaStreamSynchronize(st));
    }
    return OV_OK;
}

int ov_project_lowmodes(ov_ctx* c, int which, const ov_field* psi, int engine, double* out, void* stream)
{
    if (!c || !psi || !out) return c ? set_err(c, OV_EINVAL, "null pointer") : OV_EINVAL;
    if (which != 0 && which != 1) return set_err(c, OV_EINVAL, "which = %d (0 or 1)", which);
    EigSet& E = c->eig[which];
    if (!E.nev) return set_err(c, OV_ESTATE, "no eigenpairs stored (which=%d)", which);
    cudaStream_t st = (cudaStream_t)stream;
    const int R = psi->d.nrhs;
    const size_t ncoef = (size_t)E.nev * R;
    if (ncoef * 2 > (size_t)DSCAL_COEF) return set_err(c, OV_EINVAL, "nev * nrhs = %zu too large", ncoef);
    double2* dev = (double2*)c->dscal;
    if (engine == 1 || engine == 2) {
        OV_TRY(proj_dots_tc(c, which, psi->d, dev, st, engine));
        OV_TRY(proj_tc_status(c, st));
    } else if (engine == 0) {
        FieldDesc eta;
        const int pv = psi->d.prec;
        OV_TRY(eig_vectors(c, which, pv, st, &eta));
        const int nblk = reduce_blocks(c->g);
        const int nparts = nblk * proj_groups(R);
        OV_TRY(ensure_partials(c, nparts * ncoef * sizeof(double2)));
        OV_CUDA(c, launch_proj_dots(c->g, eta, E.nev, psi->d, (double2*)c->partials, nblk, st));
        OV_CUDA(c, launch_proj_finalize((double2*)c->partials, nparts, (int)ncoef, dev, st));
    } else {
        return set_err(c, OV_EINVAL, "engine = %d (0 CUDA cores, 1 or 2 tensor cores)", engine);
    }
    OV_CUDA(c, cudaMemcpyAsync(out, dev, ncoef * sizeof(double2), cudaMemcpyDefault, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    return OV_OK;
}

int ov_lowmode_update(ov_ctx* c, int which, const ov_field* psi, const double* coef, int engine, ov_field* out1,
                      ov_field* out2, void* stream)
{
    if (!c || !psi || !coef || !out1) return c ? set_err(c, OV_EINVAL, "null pointer") : OV_EINVAL;
    if (which != 0 && which != 1) return set_err(c, OV_EINVAL, "which = %d (0 or 1)", which);
    EigSet& E = c->eig[which];
    if (!E.nev) return set_err(c, OV_ESTATE, "no eigenpairs stored (which=%d)", which);
    const FieldDesc& pd = psi->d;
    for (const ov_field* o : {(const ov_field*)out1, (const ov_field*)out2})
        if (o && (o->d.prec != pd.prec || o->d.nrhs != pd.nrhs))
            return set_err(c, OV_EINVAL, "fields differ in precision or nrhs");
    if (out1 == psi || out2 == psi || out1 == out2) return set_err(c, OV_EINVAL, "fields must differ");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ncoef = (size_t)E.nev * pd.nrhs;
    if (ncoef * 2 > (size_t)DSCAL_COEF) return set_err(c, OV_EINVAL, "nev * nrhs = %zu too large", ncoef);
    double2* dev = (double2*)c->dscal;
    OV_CUDA(c, cudaMemcpyAsync(dev, coef, ncoef * sizeof(double2), cudaMemcpyDefault, st));
    FieldDesc o2{};
    if (out2) o2 = out2->d;
    if (engine == 1) {
        OV_TRY(proj_update_tc(c, which, pd, dev, E.d_sign, out1->d, o2, st));
        OV_TRY(proj_tc_status(c, st));
    } else if (engine == 0) {
        FieldDesc eta;
        OV_TRY(eig_vectors(c, which, pd.prec, st, &eta));
        OV_CUDA(c, launch_proj_update(c->g, eta, E.nev, dev, E.d_sign, pd, out1->d, o2, st));
    } else {
        return set_err(c, OV_EINVAL, "engine = %d (0 CUDA cores, 1 tensor cores)", engine);
    }
    OV_CUDA(c, cudaStreamSynchronize(st));
    return OV_OK;
}

long long ov_device_bytes(const ov_ctx* c) { return c ? c->bytes : -1; }

long long ov_dslash_count(const ov_ctx* c) { return c ? c->dslash_launches : -1; }

int ov_graph_stats(const ov_ctx* c, long long* captured, long long* replayed)
{
    if (!c) return OV_EINVAL;
    if (captured) *captured = c->graph_captures;
    if (replayed) *replayed = c->graph_replays;
    return OV_OK;
}

int ov_set_option(ov_ctx* c, const char* name, double value)
{
    if (!c || !name) return c ? set_err(c, OV_EINVAL, "null option name") : OV_EINVAL;
    const std::string n(name);
    if (n == "reliable_delta") {
        if (!(value > 0 && value < 1)) return set_err(c, OV_EINVAL, "reliable_delta must lie in (0, 1)");
        c->reliable_delta = value;
    } else if (n == "filter_hw" || n == "filter_dd") {
        if (value < 0 || value > 10000) return set_err(c, OV_EINVAL, "filter degree out of range");
        (n == "filter_hw" ? c->filter_hw : c->filter_dd) = (int)value;
    } else if (n == "eig_prec") {
        if (value < -1 || value >= NPREC) return set_err(c, OV_EINVAL, "eig_prec must be -1 or an ov_prec");
        c->eig_prec = (int)value;
    } else if (n == "proj_tc") {
        graphs_clear(c);
        c->proj_tc = value != 0;
    } else if (n == "net_sym") {
        c->net_sym = value != 0;
    } else if (n == "chiral") {
        c->chiral = value != 0;
    } else if (n == "rational_pass") {
        if (value != 1 && value != 2) return set_err(c, OV_EINVAL, "rational_pass must be 1 or 2");
        c->rational_pass = (int)value;
    } else if (n == "rational_tol") {
        if (!(value > 0 && value < 1)) return set_err(c, OV_EINVAL, "rational_tol must lie in (0, 1)");
        c->rational_tol = value;
    } else if (n == "clenshaw_f32") {
        graphs_clear(c);
        c->clenshaw_f32 = value != 0;
    } else if (n == "adaptive_delta") {
        if (!(value >= 0 && value < 1)) return set_err(c, OV_EINVAL, "adaptive_delta must lie in [0, 1)");
        graphs_clear(c);
        c->adaptive_delta = value;
        if (c->have_poly) set_inner_poly(c);
    } else if (n == "wait_polls") {
        if (!(value >= 0 && value <= (double)DSLASH_WAIT_POLLS))
            return set_err(c, OV_EINVAL, "wait_polls must lie in [0, %lld]", DSLASH_WAIT_POLLS);
        graphs_clear(c);
        c->wait_polls = (long long)value;
    } else if (n == "hi_prec") {
        if (value != P_F64 && value != P_DF64) return set_err(c, OV_EINVAL, "hi_prec must be OV_F64 or OV_DF64");
        c->hi_prec = (int)value;
    } else {
        return set_err(c, OV_EINVAL, "unknown option '%s'", name);
    }
    return OV_OK;
}

int ov_get_option(const ov_ctx* c, const char* name, double* value)
{
    if (!c || !name || !value) return OV_EINVAL;
    const std::string n(name);
    if (n == "reliable_delta") *value = c->reliable_delta;
    else if (n == "filter_hw") *value = c->filter_hw;
    else if (n == "filter_dd") *value = c->filter_dd;
    else if (n == "eig_prec") *value = c->eig_prec;
    else if (n == "proj_tc") *value = c->proj_tc;
    else if (n == "net_sym") *value = c->net_sym;
    else if (n == "chiral") *value = c->chiral;
    else if (n == "hi_prec") *value = c->hi_prec;
    else if (n == "wait_polls") *value = (double)c->wait_polls;
    else if (n == "adaptive_delta") *value = c->adaptive_delta;
    else if (n == "clenshaw_f32") *value = c->clenshaw_f32;
    else if (n == "rational_pass") *value = c->rational_pass;
    else if (n == "rational_tol") *value = c->rational_tol;
    else if (n == "rational_iterations") *value = (double)c->rational_iters;
    else if (n == "adaptive_degree") *value = c->degree_in;
    else if (n == "sign_delta") {
        if (c->sign_backend == 1) *value = c->rdelta;
        else if (c->coef.empty()) return OV_ESTATE;
        else *value = poly_delta(c->coef, c->eps);
    }
    else return OV_EINVAL;
    return OV_OK;
}

int ov_set_graphs(ov_ctx* c, int enable)
{
    if (!c) return OV_EINVAL;
    graphs_clear(c);
    c->use_graphs = enable != 0;
    return OV_OK;
}

int ov_set_dslash_shape(ov_ctx* c, int prec, int nrhs, int bx, int by, int variant)
{
    if (!c) return OV_EINVAL;
    OV_TRY(check_prec(c, prec));
    if (variant < 0 || variant >= DSLASH_VARIANTS || (variant >= 3 && wide(prec)) ||
        ((variant == 3 || variant == 4 || variant == 5) && by != 1))
        return set_err(c, OV_EINVAL, "bad variant %d for this precision / shape", variant);
    const int maxt = variant == 0 ? (wide(prec) ? 256 : 512) : (variant == 3 || variant >= 6 ? 128 : 256);
    if ((variant == 8 || variant == 9) && by != 1) return set_err(c, OV_EINVAL, "variants 8, 9: by must be 1");
    if (bx < 1 || by < 1 || bx * by > maxt || bx % 32) return set_err(c, OV_EINVAL, "bad shape %d x %d", bx, by);
    c->shape[{prec, nrhs}] = std::make_tuple(bx, by, variant);
    return OV_OK;
}

int ov_tune_dslash(ov_ctx* c, int prec, int nrhs, int* bx, int* by, int* variant, void* stream)
{
    if (!c) return OV_EINVAL;
    OV_TRY(check_prec(c, prec));
    if (nrhs < 1 || nrhs > 16) return set_err(c, OV_EINVAL, "nrhs out of range");
    if (!c->have_gauge) return set_err(c, OV_ESTATE, "no gauge field");
    cudaStream_t st = (cudaStream_t)stream;
    FieldDesc fi, fo;
    OV_TRY(ws_field(c, WS_IN, prec, nrhs, &fi));
    OV_TRY(ws_field(c, WS_OUT, prec, nrhs, &fo));
    OV_CUDA(c, cudaMemsetAsync(fi.data, 0, data_bytes(prec, nrhs, c->g.Vh), st));
    if (fi.norm) OV_CUDA(c, cudaMemsetAsync(fi.norm, 0, norm_bytes(prec, nrhs, c->g.Vh), st));
    // candidates: block = x sites by y right-hand sides, times the register-budget variants
    std::vector<std::tuple<int, int, int>> cand;
    for (int v = 0; v < DSLASH_VARIANTS; ++v) {
        if (v >= 3 && wide(prec)) continue;  // staged variants: FP32 arithmetic only
        if (v == 4 || v == 5) {              // bulk-copy staging: fixed 128-site blocks
            cand.push_back(std::make_tuple(128, 1, v));
            continue;
        }
        if (v == 8 || v == 9) {              // batched hop loads: 128-thread blocks, one rhs per block row
            for (int x : {64, 128}) cand.push_back(std::make_tuple(x, 1, v));
            continue;
        }
        if (v >= 6) {                        // 2 or 4 right-hand sides per thread
            const int rb = (v == 6 || v == 10) ? 2 : 4;
            if (nrhs < rb) continue;
            const int groups = (nrhs + rb - 1) / rb;
            for (int x : {32, 64, 128})
                for (int y = 1; y <= groups && x * y <= 128; ++y)
                    if (groups % y == 0 && x * y >= 64) cand.push_back(std::make_tuple(x, y, v));
            continue;
        }
        const int maxt = v == 0 ? (wide(prec) ? 256 : 512) : (v == 3 ? 128 : 256);
        for (int x : {32, 64, 128, 256})
            for (int y = 1; y <= nrhs && y <= 16; ++y) {
                if (v == 3 && y != 1) continue;
                if (nrhs % y && y != nrhs) continue;
                if (x * y > maxt || x * y < (v == 3 ? 32 : 64)) continue;
                cand.push_back(std::make_tuple(x, y, v));
            }
    }
    if (cand.empty()) cand.push_back(default_shape(prec, nrhs));
    cudaEvent_t e0, e1;
    OV_CUDA(c, cudaEventCreate(&e0));
    OV_CUDA(c, cudaEventCreate(&e1));
    float best = 1e30f;
    std::tuple<int, int, int> bsh = cand[0];
    for (auto sh : cand) {
        c->shape[{prec, nrhs}] = sh;
        OV_TRY(dslash_apply(c, fi, fo, 4.0, -0.5, 0, 0, 0, nullptr, nullptr, st));
        OV_CUDA(c, cudaEventRecord(e0, st));
        for (int i = 0; i < 10; ++i) OV_TRY(dslash_apply(c, fi, fo, 4.0, -0.5, 0, 0, 0, nullptr, nullptr, st));
        OV_CUDA(c, cudaEventRecord(e1, st));
        OV_CUDA(c, cudaEventSynchronize(e1));
        float ms = 0;
        OV_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
        if (verbose())
            fprintf(stderr, "[ov] tune prec %d nrhs %d: block %d x %d variant %d: %.2f us\n", prec, nrhs,
                    std::get<0>(sh), std::get<1>(sh), std::get<2>(sh), 100.0f * ms);
        if (ms < best) {
            best = ms;
            bsh = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->shape[{prec, nrhs}] = bsh;
    if (bx) *bx = std::get<0>(bsh);
    if (by) *by = std::get<1>(bsh);
    if (variant) *variant = std::get<2>(bsh);
    return OV_OK;
}

}  // extern "C"
