// Wilson dslash, launch variants 10-11: right-hand sides in pairs on the packed FP32 pipe.
#include "dslash_common.cuh"

namespace ov {

namespace {

// ---------------------------------------------------------------------------
// Variants 10 and 11 (multi-RHS, FP32 arithmetic, FP32 or 16-bit storage): right-hand sides in pairs
// on the packed FP32 pipe.  A thread applies D_w at one site to NP pairs of right-hand sides; each
// real of a pair's work is a float2 (the value for source 2k, the value for source 2k + 1), so the
// colour multiply, the lower-spin reconstruction and the accumulation are two-wide operations
// (fma.rn.f32x2, add.rn.f32x2, mul.rn.f32x2) whose link operand is the same in both lanes.  The link
// is loaded and its third row reconstructed once per 2 NP sources, and the arithmetic of a hop costs
// about half the instructions per source of the one-source kernels, which are bound by instruction
// issue once several sources share each link through L1.  The spin projection stays scalar: it
// writes each source's half spinor straight into its lane.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 bcast2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
// c + SG * x, SG = +1 or -1: one packed add, or one packed fused multiply-add by -1 (exact product)
template <int SG>
__device__ __forceinline__ float2 acc2(float2 c, float2 x)
{
    if constexpr (SG > 0)
        return __fadd2_rn(c, x);
    else
        return __ffma2_rn(x, make_float2(-1.f, -1.f), c);
}

// chi = U h (forward) or U^dag h (backward) for a pair of sources; the chains of link_mul, two-wide
template <int S>
__device__ __forceinline__ void link_mul_pair(const float u[18], const float2 h[12], float2 chi[12])
{
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float2 re, im;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float ur, ui;
                if constexpr (S > 0) {
                    ur = u[2 * (3 * i + j)];
                    ui = u[2 * (3 * i + j) + 1];
                } else {
                    ur = u[2 * (3 * j + i)];
                    ui = -u[2 * (3 * j + i) + 1];
                }
                const float2 hr = h[6 * a + 2 * j], hi = h[6 * a + 2 * j + 1];
                if (j == 0) {
                    re = mul2(bcast2(ur), hr);
                    im = mul2(bcast2(ur), hi);
                } else {
                    re = fma2(bcast2(ur), hr, re);
                    im = fma2(bcast2(ur), hi, im);
                }
                re = fma2(bcast2(-ui), hi, re);
                im = fma2(bcast2(ui), hr, im);
            }
            chi[6 * a + 2 * i] = re;
            chi[6 * a + 2 * i + 1] = im;
        }
    }
}

// accumulate<MU, S> for a pair of sources: upper spins += chi, lower spins -= S A_mu^dag chi
template <int MU, int S>
__device__ __forceinline__ void accumulate_pair(float2 acc[24], const float2 chi[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 x0r = chi[2 * c], x0i = chi[2 * c + 1];
        const float2 x1r = chi[6 + 2 * c], x1i = chi[6 + 2 * c + 1];
        acc[2 * c] = acc2<1>(acc[2 * c], x0r);
        acc[2 * c + 1] = acc2<1>(acc[2 * c + 1], x0i);
        acc[2 * (3 + c)] = acc2<1>(acc[2 * (3 + c)], x1r);
        acc[2 * (3 + c) + 1] = acc2<1>(acc[2 * (3 + c) + 1], x1i);
        float2* d0r = &acc[2 * (6 + c)];
        float2* d0i = &acc[2 * (6 + c) + 1];
        float2* d1r = &acc[2 * (9 + c)];
        float2* d1i = &acc[2 * (9 + c) + 1];
        // lower -= S * (A^dag chi): each term below is (sign of the A^dag entry) * (-S)
        if constexpr (MU == 0) {  // A^dag chi = (i x1, i x0): re = -x_im, im = x_re
            *d0r = acc2<S>(*d0r, x1i);
            *d0i = acc2<-S>(*d0i, x1r);
            *d1r = acc2<S>(*d1r, x0i);
            *d1i = acc2<-S>(*d1i, x0r);
        } else if constexpr (MU == 1) {  // (x1, -x0)
            *d0r = acc2<-S>(*d0r, x1r);
            *d0i = acc2<-S>(*d0i, x1i);
            *d1r = acc2<S>(*d1r, x0r);
            *d1i = acc2<S>(*d1i, x0i);
        } else if constexpr (MU == 2) {  // (i x0, -i x1)
            *d0r = acc2<S>(*d0r, x0i);
            *d0i = acc2<-S>(*d0i, x0r);
            *d1r = acc2<-S>(*d1r, x1i);
            *d1i = acc2<S>(*d1i, x1r);
        } else {  // (x0, x1)
            *d0r = acc2<-S>(*d0r, x0r);
            *d0i = acc2<-S>(*d0i, x0i);
            *d1r = acc2<-S>(*d1r, x1r);
            *d1i = acc2<-S>(*d1i, x1i);
        }
    }
}

template <int SP, int GP, int MU, int S, int NP>
__device__ __forceinline__ void hop_pair(const DslashArgs& A, const char* const in_q[2 * NP],
                                         const float* const inn_q[2 * NP], int p, int s, int sn, bool cross,
                                         float2 acc[NP][24])
{
    constexpr bool H16 = SP == P_F16 || SP == P_BF16;
    const int lpar = S > 0 ? p : 1 - p;
    const int ls = S > 0 ? s : sn;
    const char* lb = A.gauge + ((size_t)(lpar * 4 + MU) * A.g.Vh) * gauge_link_bytes_dev<GP>();
    float u[18];
    load_link<GP, float>(lb, A.g.Vh, ls, u);
    const float ph = A.g.fbc[MU];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        float va[24], vb[24], ha[12], hb[12];
        float2 h[12];
        if constexpr (H16) {
            float na = load_spinor_unscaled<SP>(in_q[2 * k], inn_q[2 * k], A.g.Vh, sn, va);
            float nb = load_spinor_unscaled<SP>(in_q[2 * k + 1], inn_q[2 * k + 1], A.g.Vh, sn, vb);
            project<MU, S, float>(va, ha);
            project<MU, S, float>(vb, hb);
            if (cross) {
                na *= ph;
                nb *= ph;
            }
            const float2 n2 = make_float2(na, nb);
#pragma unroll
            for (int i = 0; i < 12; ++i) h[i] = mul2(make_float2(ha[i], hb[i]), n2);
        } else {
            load_spinor<SP, float>(in_q[2 * k], nullptr, A.g.Vh, sn, va);
            load_spinor<SP, float>(in_q[2 * k + 1], nullptr, A.g.Vh, sn, vb);
            project<MU, S, float>(va, ha);
            project<MU, S, float>(vb, hb);
#pragma unroll
            for (int i = 0; i < 12; ++i) h[i] = make_float2(ha[i], hb[i]);
            if (cross) {
#pragma unroll
                for (int i = 0; i < 12; ++i) h[i] = mul2(h[i], bcast2(ph));
            }
        }
        float2 chi[12];
        link_mul_pair<S>(u, h, chi);
        accumulate_pair<MU, S>(acc[k], chi);
    }
}

template <int SP, int GP, int NY, int NP>
__global__ void __launch_bounds__(128) dslash_pair_kernel(DslashArgs A)
{
    constexpr int RB = 2 * NP;
    const int ngroups = ((A.nrhs + RB - 1) / RB + blockDim.y - 1) / blockDim.y;
    const BlockWork bw = block_work(ngroups);
    const int p = bw.p;
    const int s = bw.sb * blockDim.x + threadIdx.x;
    const int r0 = (bw.grp * blockDim.y + threadIdx.y) * RB;
    const Geom& g = A.g;
    if (s >= g.Vh || r0 >= A.nrhs) return;
    const int nr = A.nrhs - r0 < RB ? A.nrhs - r0 : RB;
    constexpr size_t CH = nchunk_dev<SP>() * 16;
    const size_t par_bytes = CH * g.Vh;
    const int q = 1 - p;
    const char* in_q[RB];
    const float* inn_q[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
        const int r = r0 + (j < nr ? j : 0);  // sources past the end repeat the first (never stored)
        in_q[j] = A.in + ((size_t)r * 2 + q) * par_bytes;
        inn_q[j] = A.in_n ? A.in_n + ((size_t)r * 2 + q) * g.Vh : nullptr;
    }
    int c[4];
    cb_coords(g, s, p, c);
    float2 acc[NP][24];
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[k][i] = make_float2(0.f, 0.f);
    hop_pair<SP, GP, 0, +1, NP>(A, in_q, inn_q, p, s, cb_neighbour<0>(g, s, c), c[0] + 1 == g.L[0], acc);
    hop_pair<SP, GP, 0, -1, NP>(A, in_q, inn_q, p, s, cb_neighbour<1>(g, s, c), c[0] == 0, acc);
    hop_pair<SP, GP, 1, +1, NP>(A, in_q, inn_q, p, s, cb_neighbour<2>(g, s, c), c[1] + 1 == g.L[1], acc);
    hop_pair<SP, GP, 1, -1, NP>(A, in_q, inn_q, p, s, cb_neighbour<3>(g, s, c), c[1] == 0, acc);
    hop_pair<SP, GP, 2, +1, NP>(A, in_q, inn_q, p, s, cb_neighbour<4>(g, s, c), c[2] + 1 == g.L[2], acc);
    hop_pair<SP, GP, 2, -1, NP>(A, in_q, inn_q, p, s, cb_neighbour<5>(g, s, c), c[2] == 0, acc);
    hop_pair<SP, GP, 3, +1, NP>(A, in_q, inn_q, p, s, cb_neighbour<6>(g, s, c), c[3] + 1 == g.L[3], acc);
    hop_pair<SP, GP, 3, -1, NP>(A, in_q, inn_q, p, s, cb_neighbour<7>(g, s, c), c[3] == 0, acc);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        float a0[24], a1[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            a0[i] = acc[k][i].x;
            a1[i] = acc[k][i].y;
        }
        if (2 * k < nr) epilogue<SP, NY>(A, r0 + 2 * k, p, s, a0);
        if (2 * k + 1 < nr) epilogue<SP, NY>(A, r0 + 2 * k + 1, p, s, a1);
    }
}

template <int SP, int GP, int NP>
cudaError_t launch_pair(const DslashArgs& A, int ny, dim3 block, cudaStream_t st)
{
    if constexpr (wide_dev<SP>) {
        return cudaErrorInvalidValue;
    } else {
        if ((int)(block.x * block.y) > 128) return cudaErrorInvalidValue;
        const int groups = (A.nrhs + 2 * NP - 1) / (2 * NP);
        const dim3 grid = block_grid(A.g.Vh, block.x, (groups + block.y - 1) / block.y);
        switch (ny) {
        case 0: dslash_pair_kernel<SP, GP, 0, NP><<<grid, block, 0, st>>>(A); break;
        case 1: dslash_pair_kernel<SP, GP, 1, NP><<<grid, block, 0, st>>>(A); break;
        case 2: dslash_pair_kernel<SP, GP, 2, NP><<<grid, block, 0, st>>>(A); break;
        case 3: dslash_pair_kernel<SP, GP, 3, NP><<<grid, block, 0, st>>>(A); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

struct Pair {
    template <int SP, int GP>
    static cudaError_t run(const DslashArgs& A, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
    {
        switch (var) {
        case 10: return launch_pair<SP, GP, 1>(A, ny, block, st);
        case 11: return launch_pair<SP, GP, 2>(A, ny, block, st);
        }
        return cudaErrorInvalidValue;
    }
};

}  // namespace

cudaError_t launch_dslash_pair(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
{
    return dispatch_prec<Pair>(A, sp, gp, ny, var, grid, block, st);
}

}  // namespace ov
