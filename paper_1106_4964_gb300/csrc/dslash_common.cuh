// Even/odd Wilson dslash on the internal layout (Eqs. 1-2 of the paper):
//
//   D_w(m) psi(n) = (m + 4) psi(n)
//                 - 1/2 sum_mu [ U_mu(n) (1 - gamma_mu) psi(n + mu)
//                              + U_mu(n - mu)^dag (1 + gamma_mu) psi(n - mu) ]
//
// One launch computes both parities of the output and all right-hand sides.
// Blocks are numbered with the right-hand-side group fastest, then the parity,
// then the site block (block_work below): the groups and both parities of one
// region of BX checkerboard sites run back to back, so the links and
// neighbour spinors they share are re-read from L2, not from HBM once per
// group.  Threads (x, y) of a block handle site x of right-hand side
// group * BY + y; the BY right-hand sides of a block share every link load
// through L1.
//
// Spin structure (Euclidean chiral basis, gamma_mu = [[0, A_mu], [A_mu^dag, 0]],
// A_k = -i sigma_k, A_4 = 1): (1 - S gamma_mu) psi has upper half
// h = psi_up - S A_mu psi_dn and lower half -S A_mu^dag h, so each hop
// projects to a 2-spin half spinor, multiplies it by the link and
// reconstructs the lower half (S = +1 forward, -1 backward).
//
// Generic epilogue:
//   core = a * psi(n) + b * hop_sum;  core = gamma5 core if g5_core
//   out  = core + sum_j sy[j] * y_j(n);  out = gamma5 out if g5_out
// which gives D_w (a = 4+m, b = -1/2), H_w (g5_core), and the fused
// Clenshaw step b_k = c_k psi_h + alpha H_w t + beta b_{k+1} - b_{k+2}.
//
// The kernels are split over translation units by launch variant (dslash_regs.cu: 0-2,
// dslash_staged.cu: 3-5, dslash_multi.cu: 6-7, dslash_batched.cu: 8-9, dslash_pair.cu: 10-11), so that
// they compile in parallel; this header holds what they share.
#pragma once

#include <type_traits>

#include "ov_internal.cuh"
#include "ov_kernels.h"

namespace ov {

namespace {

template <int SP>
using real_t = typename std::conditional<SP == P_F64, double, typename std::conditional<SP == P_DF64, df64, float>::type>::type;
template <int SP>
constexpr bool wide_dev = SP == P_F64 || SP == P_DF64;

template <int MU, int S, typename Real>
__device__ __forceinline__ void project(const Real v[24], Real h[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Real u0r = v[2 * (0 + c)], u0i = v[2 * (0 + c) + 1];
        Real u1r = v[2 * (3 + c)], u1i = v[2 * (3 + c) + 1];
        Real d0r = v[2 * (6 + c)], d0i = v[2 * (6 + c) + 1];
        Real d1r = v[2 * (9 + c)], d1i = v[2 * (9 + c) + 1];
        Real a0r, a0i, a1r, a1i;  // (A_mu psi_dn)_{0,1}
        if constexpr (MU == 0) {  // A = [[0,-i],[-i,0]]
            a0r = d1i; a0i = -d1r;
            a1r = d0i; a1i = -d0r;
        } else if constexpr (MU == 1) {  // A = [[0,-1],[1,0]]
            a0r = -d1r; a0i = -d1i;
            a1r = d0r; a1i = d0i;
        } else if constexpr (MU == 2) {  // A = diag(-i, i)
            a0r = d0i; a0i = -d0r;
            a1r = -d1i; a1i = d1r;
        } else {  // A = 1
            a0r = d0r; a0i = d0i;
            a1r = d1r; a1i = d1i;
        }
        h[2 * c] = u0r - S * a0r;
        h[2 * c + 1] = u0i - S * a0i;
        h[6 + 2 * c] = u1r - S * a1r;
        h[6 + 2 * c + 1] = u1i - S * a1i;
    }
}

template <int MU, int S, typename Real>
__device__ __forceinline__ void accumulate(Real acc[24], const Real chi[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Real x0r = chi[2 * c], x0i = chi[2 * c + 1];
        Real x1r = chi[6 + 2 * c], x1i = chi[6 + 2 * c + 1];
        acc[2 * (0 + c)] += x0r;
        acc[2 * (0 + c) + 1] += x0i;
        acc[2 * (3 + c)] += x1r;
        acc[2 * (3 + c) + 1] += x1i;
        Real b0r, b0i, b1r, b1i;  // (A_mu^dag chi)_{0,1}
        if constexpr (MU == 0) {  // A^dag = [[0,i],[i,0]]
            b0r = -x1i; b0i = x1r;
            b1r = -x0i; b1i = x0r;
        } else if constexpr (MU == 1) {  // A^dag = [[0,1],[-1,0]]
            b0r = x1r; b0i = x1i;
            b1r = -x0r; b1i = -x0i;
        } else if constexpr (MU == 2) {  // A^dag = diag(i, -i)
            b0r = -x0i; b0i = x0r;
            b1r = x1i; b1i = -x1r;
        } else {
            b0r = x0r; b0i = x0i;
            b1r = x1r; b1i = x1i;
        }
        acc[2 * (6 + c)] -= S * b0r;
        acc[2 * (6 + c) + 1] -= S * b0i;
        acc[2 * (9 + c)] -= S * b1r;
        acc[2 * (9 + c) + 1] -= S * b1i;
    }
}

// a * b + c as one fused multiply-add (FP32, FP64); double-float composes its own operations
template <typename Real>
__device__ __forceinline__ Real fmac(Real a, Real b, Real c)
{
    if constexpr (std::is_same<Real, df64>::value)
        return a * b + c;
    else
        return fma(a, b, c);
}

// chi = U h (forward) or U^dag h (backward), two spins.  Each real part is one chain of fused
// multiply-adds, 6 per component (the form re += ur*hr - ui*hi would cost a multiply, a fused
// multiply-add and an add per term: 108 instead of 72 operations per hop)
template <int S, typename Real>
__device__ __forceinline__ void link_mul(const Real u[18], const Real h[12], Real chi[12])
{
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Real re, im;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                Real ur, ui;  // U_ij, or conj(U_ji) for the backward hop
                if constexpr (S > 0) {
                    ur = u[2 * (3 * i + j)];
                    ui = u[2 * (3 * i + j) + 1];
                } else {
                    ur = u[2 * (3 * j + i)];
                    ui = -u[2 * (3 * j + i) + 1];
                }
                const Real hr = h[6 * a + 2 * j], hi = h[6 * a + 2 * j + 1];
                if (j == 0) {
                    re = ur * hr;
                    im = ur * hi;
                } else {
                    re = fmac<Real>(ur, hr, re);
                    im = fmac<Real>(ur, hi, im);
                }
                re = fmac<Real>(-ui, hi, re);
                im = fmac<Real>(ui, hr, im);
            }
            chi[6 * a + 2 * i] = re;
            chi[6 * a + 2 * i + 1] = im;
        }
    }
}

template <int SP, int GP, int MU, int S>
__device__ __forceinline__ void hop(const DslashArgs& A, const char* in_q, const float* inn_q, int p, int s, int sn,
                                    bool cross, real_t<SP> acc[24])
{
    using Real = real_t<SP>;
    Real v[24];
    Real h[12];
    if constexpr (SP == P_F16 || SP == P_BF16) {
        // 16-bit storage: project the unscaled values and apply the site's scale (and the boundary
        // phase) to the 12 projected reals instead of the 24 loaded ones
        float n = load_spinor_unscaled<SP>(in_q, inn_q, A.g.Vh, sn, v);
        project<MU, S, Real>(v, h);
        if (cross) n *= A.g.fbc[MU];
#pragma unroll
        for (int i = 0; i < 12; ++i) h[i] *= n;
    } else {
        load_spinor<SP, Real>(in_q, inn_q, A.g.Vh, sn, v);
        project<MU, S, Real>(v, h);
        if (cross) {
            const Real ph = coef<Real>(A.g.bc[MU], A.g.fbc[MU]);
#pragma unroll
            for (int i = 0; i < 12; ++i) h[i] *= ph;
        }
    }
    const int lpar = S > 0 ? p : 1 - p;
    const int ls = S > 0 ? s : sn;
    const char* lb = A.gauge + ((size_t)(lpar * 4 + MU) * A.g.Vh) * gauge_link_bytes_dev<GP>();
    Real u[18];
    load_link<GP, Real>(lb, A.g.Vh, ls, u);
    Real chi[12];
    link_mul<S, Real>(u, h, chi);
    accumulate<MU, S, Real>(acc, chi);
}

template <int SP, int NY>
__device__ __forceinline__ void epilogue(const DslashArgs& A, int r, int p, int s, const real_t<SP> acc[24]);

// Register-budget variants chosen by the autotuner: VAR 0 lets the compiler
// use what it wants (low occupancy, long latency chains), VAR 1 and 2 cap
// the registers so that more warps are resident to hide load latency.
template <int SP, int VAR>
struct Bounds {
    static constexpr int maxt = VAR == 0 ? (wide_dev<SP> ? 256 : 512) : 256;
    static constexpr int minb = VAR == 0 ? 1 : (wide_dev<SP> ? VAR + 1 : VAR + 2);
};

// The work of block blockIdx.x in a launch of `ngroups` right-hand-side groups: parity p, site block sb,
// group grp (grid: 2 x site blocks x ngroups, one dimension)
struct BlockWork {
    int p, sb, grp;
};
__device__ __forceinline__ BlockWork block_work(int ngroups)
{
    const int b = (int)blockIdx.x;
    if (ngroups == 1) return {b & 1, b >> 1, 0};
    const int rest = b / ngroups;
    return {rest & 1, rest >> 1, b - rest * ngroups};
}

template <int SP, int GP, int NY, int VAR>
__global__ void __launch_bounds__(Bounds<SP, VAR>::maxt, Bounds<SP, VAR>::minb) dslash_kernel(DslashArgs A)
{
    using Real = real_t<SP>;
    const BlockWork bw = block_work((A.nrhs + blockDim.y - 1) / blockDim.y);
    const int p = bw.p;
    const int s = bw.sb * blockDim.x + threadIdx.x;
    const int r = bw.grp * blockDim.y + threadIdx.y;
    const Geom& g = A.g;
    if (s >= g.Vh || r >= A.nrhs) return;

    constexpr size_t CH = nchunk_dev<SP>() * 16;
    const size_t par_bytes = CH * g.Vh;
    const int q = 1 - p;
    const char* in_q = A.in + ((size_t)r * 2 + q) * par_bytes;
    const float* inn_q = A.in_n ? A.in_n + ((size_t)r * 2 + q) * g.Vh : nullptr;

    int c[4];
    cb_coords(g, s, p, c);
    Real acc[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) acc[i] = 0;

    // neighbour index computed at its hop (short live ranges); the flag marks a boundary crossing
    hop<SP, GP, 0, +1>(A, in_q, inn_q, p, s, cb_neighbour<0>(g, s, c), c[0] + 1 == g.L[0], acc);
    hop<SP, GP, 0, -1>(A, in_q, inn_q, p, s, cb_neighbour<1>(g, s, c), c[0] == 0, acc);
    hop<SP, GP, 1, +1>(A, in_q, inn_q, p, s, cb_neighbour<2>(g, s, c), c[1] + 1 == g.L[1], acc);
    hop<SP, GP, 1, -1>(A, in_q, inn_q, p, s, cb_neighbour<3>(g, s, c), c[1] == 0, acc);
    hop<SP, GP, 2, +1>(A, in_q, inn_q, p, s, cb_neighbour<4>(g, s, c), c[2] + 1 == g.L[2], acc);
    hop<SP, GP, 2, -1>(A, in_q, inn_q, p, s, cb_neighbour<5>(g, s, c), c[2] == 0, acc);
    hop<SP, GP, 3, +1>(A, in_q, inn_q, p, s, cb_neighbour<6>(g, s, c), c[3] + 1 == g.L[3], acc);
    hop<SP, GP, 3, -1>(A, in_q, inn_q, p, s, cb_neighbour<7>(g, s, c), c[3] == 0, acc);

    epilogue<SP, NY>(A, r, p, s, acc);
}

// out(n) = g5_out[ g5_core(a psi(n) + b acc) + sum_j sy_j y_j(n) ], stored in the field format
template <int SP, int NY>
__device__ __forceinline__ void epilogue(const DslashArgs& A, int r, int p, int s, const real_t<SP> acc[24])
{
    using Real = real_t<SP>;
    const Geom& g = A.g;
    constexpr size_t CH = nchunk_dev<SP>() * 16;
    const size_t par_bytes = CH * g.Vh;
    const size_t off = ((size_t)r * 2 + p) * par_bytes;
    const size_t noff = ((size_t)r * 2 + p) * g.Vh;
    Real o[24];
    {
        Real self[24];
        load_spinor<SP, Real>(A.in + off, A.in_n ? A.in_n + noff : nullptr, g.Vh, s, self);
        const Real a = coef<Real>(A.a, A.fa), b = coef<Real>(A.b, A.fb);
#pragma unroll
        for (int i = 0; i < 24; ++i) o[i] = a * self[i] + b * acc[i];
    }
    if (A.g5_core) {
#pragma unroll
        for (int i = 12; i < 24; ++i) o[i] = -o[i];
    }
#pragma unroll
    for (int j = 0; j < NY; ++j) {
        Real w[24];
        load_spinor<SP, Real>(A.y[j] + off, A.y_n[j] ? A.y_n[j] + noff : nullptr, g.Vh, s, w);
        const Real sj = coef<Real>(A.sy[j], A.fsy[j]);
#pragma unroll
        for (int i = 0; i < 24; ++i) o[i] += sj * w[i];
    }
    if (A.g5_out) {
#pragma unroll
        for (int i = 12; i < 24; ++i) o[i] = -o[i];
    }
    store_spinor<SP, Real>(A.out + off, A.out_n ? A.out_n + noff : nullptr, g.Vh, s, o);
}

// Host side of block_work: the one-dimensional grid of a launch with site blocks of bx sites
inline dim3 block_grid(int Vh, int bx, int ngroups)
{
    return dim3((unsigned)(2 * ((Vh + bx - 1) / bx) * ngroups));
}

// One launcher per precision pair: G::run<SP, GP> for the seven supported (spinor, link) formats.
template <class G>
cudaError_t dispatch_prec(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block,
                          cudaStream_t st)
{
    if (sp == P_F64 && gp == P_F64) return G::template run<P_F64, P_F64>(A, ny, var, grid, block, st);
    if (sp == P_DF64 && gp == P_DF64) return G::template run<P_DF64, P_DF64>(A, ny, var, grid, block, st);
    if (sp == P_F32 && gp == P_F32) return G::template run<P_F32, P_F32>(A, ny, var, grid, block, st);
    if (sp == P_F16 && gp == P_F16) return G::template run<P_F16, P_F16>(A, ny, var, grid, block, st);
    if (sp == P_BF16 && gp == P_BF16) return G::template run<P_BF16, P_BF16>(A, ny, var, grid, block, st);
    if (sp == P_F32 && gp == P_F16) return G::template run<P_F32, P_F16>(A, ny, var, grid, block, st);
    if (sp == P_F32 && gp == P_BF16) return G::template run<P_F32, P_BF16>(A, ny, var, grid, block, st);
    return cudaErrorInvalidValue;
}

}  // namespace

}  // namespace ov
