// Wilson dslash, launch variants 6-7: several right-hand sides per thread.
#include "dslash_common.cuh"

namespace ov {

namespace {

// ---------------------------------------------------------------------------
// Variants 6 and 7 (multi-RHS, FP32 arithmetic): each thread applies D_w at one
// site to RB = 2 or 4 right-hand sides, so every link is loaded and its third
// row reconstructed once per RB right-hand sides instead of once per
// right-hand side (the multi-RHS launch is bound by instruction issue, and the
// link work is a fifth of it).  Threads (x, y): site x of the block's range,
// right-hand sides RB * (group * BY + y) + j, j < RB (block_work numbers the groups).
// ---------------------------------------------------------------------------
template <int SP, int GP, int MU, int S, int RB>
__device__ __forceinline__ void hop_multi(const DslashArgs& A, const char* const in_q[RB], const float* const inn_q[RB],
                                          int nr, int p, int s, int sn, bool cross, float acc[RB][24])
{
    const int lpar = S > 0 ? p : 1 - p;
    const int ls = S > 0 ? s : sn;
    const char* lb = A.gauge + ((size_t)(lpar * 4 + MU) * A.g.Vh) * gauge_link_bytes_dev<GP>();
    float u[18];
    load_link<GP, float>(lb, A.g.Vh, ls, u);
    const float ph = cross ? A.g.fbc[MU] : 1.f;
#pragma unroll
    for (int j = 0; j < RB; ++j) {
        if (j < nr) {
            float v[24];
            load_spinor<SP, float>(in_q[j], inn_q[j], A.g.Vh, sn, v);
            float h[12];
            project<MU, S, float>(v, h);
#pragma unroll
            for (int i = 0; i < 12; ++i) h[i] *= ph;
            float chi[12];
            link_mul<S, float>(u, h, chi);
            accumulate<MU, S, float>(acc[j], chi);
        }
    }
}

template <int SP, int GP, int NY, int RB>
__global__ void __launch_bounds__(128) dslash_multi_kernel(DslashArgs A)
{
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
        const int r = r0 + (j < nr ? j : 0);
        in_q[j] = A.in + ((size_t)r * 2 + q) * par_bytes;
        inn_q[j] = A.in_n ? A.in_n + ((size_t)r * 2 + q) * g.Vh : nullptr;
    }
    int c[4];
    cb_coords(g, s, p, c);
    float acc[RB][24];
#pragma unroll
    for (int j = 0; j < RB; ++j)
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[j][i] = 0.f;
    hop_multi<SP, GP, 0, +1, RB>(A, in_q, inn_q, nr, p, s, cb_neighbour<0>(g, s, c), c[0] + 1 == g.L[0], acc);
    hop_multi<SP, GP, 0, -1, RB>(A, in_q, inn_q, nr, p, s, cb_neighbour<1>(g, s, c), c[0] == 0, acc);
    hop_multi<SP, GP, 1, +1, RB>(A, in_q, inn_q, nr, p, s, cb_neighbour<2>(g, s, c), c[1] + 1 == g.L[1], acc);
    hop_multi<SP, GP, 1, -1, RB>(A, in_q, inn_q, nr, p, s, cb_neighbour<3>(g, s, c), c[1] == 0, acc);
    hop_multi<SP, GP, 2, +1, RB>(A, in_q, inn_q, nr, p, s, cb_neighbour<4>(g, s, c), c[2] + 1 == g.L[2], acc);
    hop_multi<SP, GP, 2, -1, RB>(A, in_q, inn_q, nr, p, s, cb_neighbour<5>(g, s, c), c[2] == 0, acc);
    hop_multi<SP, GP, 3, +1, RB>(A, in_q, inn_q, nr, p, s, cb_neighbour<6>(g, s, c), c[3] + 1 == g.L[3], acc);
    hop_multi<SP, GP, 3, -1, RB>(A, in_q, inn_q, nr, p, s, cb_neighbour<7>(g, s, c), c[3] == 0, acc);
#pragma unroll
    for (int j = 0; j < RB; ++j)
        if (j < nr) epilogue<SP, NY>(A, r0 + j, p, s, acc[j]);
}

template <int SP, int GP, int RB>
cudaError_t launch_multi(const DslashArgs& A, int ny, dim3 block, cudaStream_t st)
{
    if constexpr (wide_dev<SP>) {
        return cudaErrorInvalidValue;
    } else {
        if ((int)(block.x * block.y) > 128) return cudaErrorInvalidValue;
        const int groups = (A.nrhs + RB - 1) / RB;
        const dim3 grid = block_grid(A.g.Vh, block.x, (groups + block.y - 1) / block.y);
        switch (ny) {
        case 0: dslash_multi_kernel<SP, GP, 0, RB><<<grid, block, 0, st>>>(A); break;
        case 1: dslash_multi_kernel<SP, GP, 1, RB><<<grid, block, 0, st>>>(A); break;
        case 2: dslash_multi_kernel<SP, GP, 2, RB><<<grid, block, 0, st>>>(A); break;
        case 3: dslash_multi_kernel<SP, GP, 3, RB><<<grid, block, 0, st>>>(A); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

struct Multi {
    template <int SP, int GP>
    static cudaError_t run(const DslashArgs& A, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
    {
        switch (var) {
        case 6: return launch_multi<SP, GP, 2>(A, ny, block, st);
        case 7: return launch_multi<SP, GP, 4>(A, ny, block, st);
        }
        return cudaErrorInvalidValue;
    }
};

}  // namespace

cudaError_t launch_dslash_multi(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
{
    return dispatch_prec<Multi>(A, sp, gp, ny, var, grid, block, st);
}

}  // namespace ov
