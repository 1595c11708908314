// Wilson dslash, launch variants 8-9: hop loads batched ahead of their arithmetic.
#include "dslash_common.cuh"

namespace ov {

namespace {

// ---------------------------------------------------------------------------
// Variants 8 and 9 (FP32 arithmetic; FP32 or 16-bit storage): batched loads.  The loads of NB hops
// (neighbour spinor, its scale and the link rows, kept in their storage format) are all issued before
// any of those hops is computed, so a thread has NB hops of memory requests in flight instead of one;
// the kernel trades occupancy (more registers per thread) for memory-level parallelism per warp.
// NB = 4: two groups of four hops (forward and backward of x, y, then of z, t); NB = 8: all eight.
// ---------------------------------------------------------------------------
template <int SP, int GP>
struct RawHop {
    static constexpr bool H16 = SP == P_F16 || SP == P_BF16;
    static constexpr bool L16 = GP == P_F16 || GP == P_BF16;
    uint4 sp[H16 ? 3 : 6];   // spinor chunks (16-bit halves or FP32)
    float n;                 // 16-bit site scale
    uint4 lk32[L16 ? 1 : 3]; // FP32 link rows
    uint2 lk16[L16 ? 3 : 1]; // 16-bit link rows
};

template <int SP, int GP>
__device__ __forceinline__ void raw_load(RawHop<SP, GP>& R, const char* in_q, const float* inn_q, int Vh, int sn,
                                         const char* lb, int ls)
{
    const uint4* b = reinterpret_cast<const uint4*>(in_q);
#pragma unroll
    for (int k = 0; k < (RawHop<SP, GP>::H16 ? 3 : 6); ++k) R.sp[k] = __ldg(b + (size_t)k * Vh + sn);
    if constexpr (RawHop<SP, GP>::H16) R.n = __ldg(inn_q + sn);
    if constexpr (RawHop<SP, GP>::L16) {
        const uint2* l = reinterpret_cast<const uint2*>(lb);
#pragma unroll
        for (int k = 0; k < 3; ++k) R.lk16[k] = __ldg(l + (size_t)k * Vh + ls);
    } else {
        const uint4* l = reinterpret_cast<const uint4*>(lb);
#pragma unroll
        for (int k = 0; k < 3; ++k) R.lk32[k] = __ldg(l + (size_t)k * Vh + ls);
    }
}

template <int SP, int GP, int MU, int S>
__device__ __forceinline__ void raw_hop(const RawHop<SP, GP>& R, bool cross, float phase, float acc[24])
{
    float v[24];
    float scale = 1.f;
    if constexpr (RawHop<SP, GP>::H16) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 a0 = Half<SP>::to2(R.sp[k].x), a1 = Half<SP>::to2(R.sp[k].y), a2 = Half<SP>::to2(R.sp[k].z),
                         a3 = Half<SP>::to2(R.sp[k].w);
            v[8 * k + 0] = a0.x;
            v[8 * k + 1] = a0.y;
            v[8 * k + 2] = a1.x;
            v[8 * k + 3] = a1.y;
            v[8 * k + 4] = a2.x;
            v[8 * k + 5] = a2.y;
            v[8 * k + 6] = a3.x;
            v[8 * k + 7] = a3.y;
        }
        scale = R.n;
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            v[4 * k] = __uint_as_float(R.sp[k].x);
            v[4 * k + 1] = __uint_as_float(R.sp[k].y);
            v[4 * k + 2] = __uint_as_float(R.sp[k].z);
            v[4 * k + 3] = __uint_as_float(R.sp[k].w);
        }
    }
    float h[12];
    project<MU, S, float>(v, h);
    if (cross) scale *= phase;
    if (RawHop<SP, GP>::H16 || cross) {
#pragma unroll
        for (int i = 0; i < 12; ++i) h[i] *= scale;
    }
    float u[18];
    if constexpr (RawHop<SP, GP>::L16) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 a0 = Half<GP>::to2(R.lk16[k].x), a1 = Half<GP>::to2(R.lk16[k].y);
            u[4 * k] = a0.x;
            u[4 * k + 1] = a0.y;
            u[4 * k + 2] = a1.x;
            u[4 * k + 3] = a1.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            u[4 * k] = __uint_as_float(R.lk32[k].x);
            u[4 * k + 1] = __uint_as_float(R.lk32[k].y);
            u[4 * k + 2] = __uint_as_float(R.lk32[k].z);
            u[4 * k + 3] = __uint_as_float(R.lk32[k].w);
        }
    }
    link_row2<float>(u);
    float chi[12];
    link_mul<S, float>(u, h, chi);
    accumulate<MU, S, float>(acc, chi);
}

template <int SP, int GP, int NY, int NB>
__global__ void __launch_bounds__(128) dslash_batched_kernel(DslashArgs A)
{
    const BlockWork bw = block_work((A.nrhs + blockDim.y - 1) / blockDim.y);
    const int p = bw.p;
    const int s = bw.sb * blockDim.x + threadIdx.x;
    const int r = bw.grp * blockDim.y + threadIdx.y;
    const Geom& g = A.g;
    if (s >= g.Vh || r >= A.nrhs) return;
    constexpr size_t CH = nchunk_dev<SP>() * 16;
    constexpr size_t LB = gauge_link_bytes_dev<GP>();
    const size_t par_bytes = CH * g.Vh;
    const int q = 1 - p;
    const char* in_q = A.in + ((size_t)r * 2 + q) * par_bytes;
    const float* inn_q = A.in_n ? A.in_n + ((size_t)r * 2 + q) * g.Vh : nullptr;
    int c[4];
    cb_coords(g, s, p, c);
    int nb[8];
    cb_neighbours(g, s, c, nb);
    const bool cr[8] = {c[0] + 1 == g.L[0], c[0] == 0, c[1] + 1 == g.L[1], c[1] == 0,
                        c[2] + 1 == g.L[2], c[2] == 0, c[3] + 1 == g.L[3], c[3] == 0};
    // link of hop h: forward U_mu(n) at (p, s); backward U_mu(n - mu) at (q, neighbour)
    auto lbase = [&](int h) {
        const int mu = h >> 1;
        const int lpar = (h & 1) ? q : p;
        return A.gauge + ((size_t)(lpar * 4 + mu) * g.Vh) * LB;
    };
    float acc[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) acc[i] = 0.f;
    RawHop<SP, GP> R[NB];
#pragma unroll
    for (int g0 = 0; g0 < 8; g0 += NB) {
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int h = g0 + j;
            raw_load<SP, GP>(R[j], in_q, inn_q, g.Vh, nb[h], lbase(h), (h & 1) ? nb[h] : s);
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int h = g0 + j;
            switch (h) {
            case 0: raw_hop<SP, GP, 0, +1>(R[j], cr[0], g.fbc[0], acc); break;
            case 1: raw_hop<SP, GP, 0, -1>(R[j], cr[1], g.fbc[0], acc); break;
            case 2: raw_hop<SP, GP, 1, +1>(R[j], cr[2], g.fbc[1], acc); break;
            case 3: raw_hop<SP, GP, 1, -1>(R[j], cr[3], g.fbc[1], acc); break;
            case 4: raw_hop<SP, GP, 2, +1>(R[j], cr[4], g.fbc[2], acc); break;
            case 5: raw_hop<SP, GP, 2, -1>(R[j], cr[5], g.fbc[2], acc); break;
            case 6: raw_hop<SP, GP, 3, +1>(R[j], cr[6], g.fbc[3], acc); break;
            default: raw_hop<SP, GP, 3, -1>(R[j], cr[7], g.fbc[3], acc); break;
            }
        }
    }
    epilogue<SP, NY>(A, r, p, s, acc);
}

template <int SP, int GP, int NB>
cudaError_t launch_batched(const DslashArgs& A, int ny, dim3 grid, dim3 block, cudaStream_t st)
{
    if constexpr (wide_dev<SP>) {
        return cudaErrorInvalidValue;
    } else {
        if ((int)(block.x * block.y) > 128) return cudaErrorInvalidValue;
        switch (ny) {
        case 0: dslash_batched_kernel<SP, GP, 0, NB><<<grid, block, 0, st>>>(A); break;
        case 1: dslash_batched_kernel<SP, GP, 1, NB><<<grid, block, 0, st>>>(A); break;
        case 2: dslash_batched_kernel<SP, GP, 2, NB><<<grid, block, 0, st>>>(A); break;
        case 3: dslash_batched_kernel<SP, GP, 3, NB><<<grid, block, 0, st>>>(A); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

struct Batched {
    template <int SP, int GP>
    static cudaError_t run(const DslashArgs& A, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
    {
        switch (var) {
        case 8: return launch_batched<SP, GP, 4>(A, ny, grid, block, st);
        case 9: return launch_batched<SP, GP, 8>(A, ny, grid, block, st);
        }
        return cudaErrorInvalidValue;
    }
};

}  // namespace

cudaError_t launch_dslash_batched(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
{
    return dispatch_prec<Batched>(A, sp, gp, ny, var, grid, block, st);
}

}  // namespace ov
