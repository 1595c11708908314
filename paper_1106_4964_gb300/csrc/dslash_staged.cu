// Wilson dslash, launch variants 3-5: neighbour spinors staged in shared memory.
#include "dslash_common.cuh"

namespace ov {

namespace {

// ---------------------------------------------------------------------------
// Variant 3 (FP32 arithmetic only): every thread stages the 8 neighbour
// spinors and links of its site into its own shared-memory slots with
// cp.async, one commit group per hop, so all of a site's loads are in flight
// at once without occupying registers; hop h then waits only for group h.
// Slots are chunk-major ([hop][chunk][thread]) so a warp's accesses hit
// consecutive 16-byte words.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int SP, int GP>
struct AsyncLayout {
    static constexpr int SCH = nchunk_dev<SP>();                  // 16-byte spinor chunks
    static constexpr int LCB = GP == P_F32 ? 16 : 8;              // bytes of each of the 3 link chunks
    static constexpr int NRM = (SP == P_F16 || SP == P_BF16) ? 4 : 0;
    static constexpr int PER_THREAD = 8 * (SCH * 16 + 3 * LCB + NRM);
    __device__ static uint8_t* spin(uint8_t* sm, int BX, int h, int k, int t) { return sm + ((h * SCH + k) * BX + t) * 16; }
    __device__ static uint8_t* link(uint8_t* sm, int BX, int h, int k, int t)
    {
        return sm + 8 * SCH * 16 * BX + ((h * 3 + k) * BX + t) * LCB;
    }
    __device__ static uint8_t* norm(uint8_t* sm, int BX, int h, int t)
    {
        return sm + 8 * (SCH * 16 + 3 * LCB) * BX + (h * BX + t) * 4;
    }
};

template <int SP, int GP>
__device__ __forceinline__ void stage_hop(uint8_t* sm, int BX, int t, int h, const char* in_q, const float* inn_q,
                                          int Vh, int sn, const char* lbase, int ls)
{
    using L = AsyncLayout<SP, GP>;
#pragma unroll
    for (int k = 0; k < L::SCH; ++k) cp_async16(L::spin(sm, BX, h, k, t), in_q + ((size_t)k * Vh + sn) * 16);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if constexpr (L::LCB == 16)
            cp_async16(L::link(sm, BX, h, k, t), lbase + ((size_t)k * Vh + ls) * 16);
        else
            cp_async8(L::link(sm, BX, h, k, t), lbase + ((size_t)k * Vh + ls) * 8);
    }
    if constexpr (L::NRM) cp_async4(L::norm(sm, BX, h, t), inn_q + sn);
    cp_async_commit();
}

template <int SP, int GP, int MU, int S, int H>
__device__ __forceinline__ void hop_staged(uint8_t* sm, int BX, int t, bool cross, float phase, float acc[24])
{
    using L = AsyncLayout<SP, GP>;
    cp_async_wait<7 - H>();
    float v[24];
    if constexpr (SP == P_F32) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(L::spin(sm, BX, H, k, t));
            v[4 * k] = a.x;
            v[4 * k + 1] = a.y;
            v[4 * k + 2] = a.z;
            v[4 * k + 3] = a.w;
        }
    } else {
        const float n = *reinterpret_cast<const float*>(L::norm(sm, BX, H, t));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 a = *reinterpret_cast<const uint4*>(L::spin(sm, BX, H, k, t));
            const float2 a0 = Half<SP>::to2(a.x), a1 = Half<SP>::to2(a.y), a2 = Half<SP>::to2(a.z),
                         a3 = Half<SP>::to2(a.w);
            v[8 * k + 0] = a0.x * n;
            v[8 * k + 1] = a0.y * n;
            v[8 * k + 2] = a1.x * n;
            v[8 * k + 3] = a1.y * n;
            v[8 * k + 4] = a2.x * n;
            v[8 * k + 5] = a2.y * n;
            v[8 * k + 6] = a3.x * n;
            v[8 * k + 7] = a3.y * n;
        }
    }
    float h[12];
    project<MU, S, float>(v, h);
    if (cross) {
#pragma unroll
        for (int i = 0; i < 12; ++i) h[i] *= phase;
    }
    float u[18];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if constexpr (GP == P_F32) {
            const float4 a = *reinterpret_cast<const float4*>(L::link(sm, BX, H, k, t));
            u[4 * k] = a.x;
            u[4 * k + 1] = a.y;
            u[4 * k + 2] = a.z;
            u[4 * k + 3] = a.w;
        } else {
            const uint2 a = *reinterpret_cast<const uint2*>(L::link(sm, BX, H, k, t));
            const float2 a0 = Half<GP>::to2(a.x), a1 = Half<GP>::to2(a.y);
            u[4 * k] = a0.x;
            u[4 * k + 1] = a0.y;
            u[4 * k + 2] = a1.x;
            u[4 * k + 3] = a1.y;
        }
    }
    link_row2<float>(u);  // row 2 = conj(row0 x row1)
    float chi[12];
    link_mul<S, float>(u, h, chi);
    accumulate<MU, S, float>(acc, chi);
}

template <int SP, int GP, int NY>
__global__ void __launch_bounds__(128) dslash_staged_kernel(DslashArgs A)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const int BX = blockDim.x, tx = threadIdx.x;
    const BlockWork bw = block_work(A.nrhs);  // one right-hand side per block
    const int p = bw.p;
    const int s = bw.sb * BX + tx;
    const int r = bw.grp;
    const Geom& g = A.g;
    if (s >= g.Vh || r >= A.nrhs) return;
    constexpr size_t CH = nchunk_dev<SP>() * 16;
    const size_t par_bytes = CH * g.Vh;
    const int q = 1 - p;
    const char* in_q = A.in + ((size_t)r * 2 + q) * par_bytes;
    const float* inn_q = A.in_n ? A.in_n + ((size_t)r * 2 + q) * g.Vh : nullptr;
    int c[4];
    cb_coords(g, s, p, c);
    int nbr[8];
    cb_neighbours(g, s, c, nbr);
    // hops crossing the lattice boundary (they carry the boundary phase)
    const bool xp0 = c[0] + 1 == g.L[0], xm0 = c[0] == 0, yp0 = c[1] + 1 == g.L[1], ym0 = c[1] == 0;
    const bool zp0 = c[2] + 1 == g.L[2], zm0 = c[2] == 0, tp0 = c[3] + 1 == g.L[3], tm0 = c[3] == 0;
    const int* sn = nbr;
    constexpr size_t LB = gauge_link_bytes_dev<GP>();
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        const int mu = h >> 1;
        const bool fwd = (h & 1) == 0;
        const int lpar = fwd ? p : q, ls = fwd ? s : sn[h];
        stage_hop<SP, GP>(sm, BX, tx, h, in_q, inn_q, g.Vh, sn[h], A.gauge + ((size_t)(lpar * 4 + mu) * g.Vh) * LB, ls);
    }
    float acc[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) acc[i] = 0.f;
    hop_staged<SP, GP, 0, +1, 0>(sm, BX, tx, xp0, g.fbc[0], acc);
    hop_staged<SP, GP, 0, -1, 1>(sm, BX, tx, xm0, g.fbc[0], acc);
    hop_staged<SP, GP, 1, +1, 2>(sm, BX, tx, yp0, g.fbc[1], acc);
    hop_staged<SP, GP, 1, -1, 3>(sm, BX, tx, ym0, g.fbc[1], acc);
    hop_staged<SP, GP, 2, +1, 4>(sm, BX, tx, zp0, g.fbc[2], acc);
    hop_staged<SP, GP, 2, -1, 5>(sm, BX, tx, zm0, g.fbc[2], acc);
    hop_staged<SP, GP, 3, +1, 6>(sm, BX, tx, tp0, g.fbc[3], acc);
    hop_staged<SP, GP, 3, -1, 7>(sm, BX, tx, tm0, g.fbc[3], acc);
    epilogue<SP, NY>(A, r, p, s, acc);
}

template <int SP, int GP>
cudaError_t launch_staged(const DslashArgs& A, int ny, dim3 grid, dim3 block, cudaStream_t st)
{
    if constexpr (wide_dev<SP>) {
        return cudaErrorInvalidValue;
    } else {
        if (block.y != 1 || block.x > 128) return cudaErrorInvalidValue;
        const size_t shm = (size_t)block.x * AsyncLayout<SP, GP>::PER_THREAD;
        static bool attr_set[4] = {false, false, false, false};
        if (!attr_set[ny]) {
            cudaError_t e = cudaSuccess;
            switch (ny) {
            case 0: e = cudaFuncSetAttribute(dslash_staged_kernel<SP, GP, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024); break;
            case 1: e = cudaFuncSetAttribute(dslash_staged_kernel<SP, GP, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024); break;
            case 2: e = cudaFuncSetAttribute(dslash_staged_kernel<SP, GP, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024); break;
            case 3: e = cudaFuncSetAttribute(dslash_staged_kernel<SP, GP, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024); break;
            default: return cudaErrorInvalidValue;
            }
            if (e != cudaSuccess) return e;
            attr_set[ny] = true;
        }
        const dim3 g2 = block_grid(A.g.Vh, block.x, A.nrhs);
        switch (ny) {
        case 0: dslash_staged_kernel<SP, GP, 0><<<g2, block, shm, st>>>(A); break;
        case 1: dslash_staged_kernel<SP, GP, 1><<<g2, block, shm, st>>>(A); break;
        case 2: dslash_staged_kernel<SP, GP, 2><<<g2, block, shm, st>>>(A); break;
        case 3: dslash_staged_kernel<SP, GP, 3><<<g2, block, shm, st>>>(A); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

// ---------------------------------------------------------------------------
// Variant 4 (FP32 arithmetic, FP32 or 16-bit storage): neighbour spinors
// staged in shared memory by the bulk-copy engine (1-D TMA).  A block owns
// TB consecutive checkerboard sites [s0, s0 + TB) of one parity and one
// right-hand side; the neighbours of the other parity lie in five index
// ranges, [s0 - Lxh - 1, s0 + TB + Lxh + 1) for the x and y hops and the
// ranges shifted by +-Lxh Ly (z hops) and +-Lxh Ly Lz (t hops).  Thread 0
// issues one cp.async.bulk per (range, chunk) plus the per-site scales of
// 16-bit storage, all completing on one mbarrier; a hop whose neighbour lies
// outside its range (lattice wrap-around, clipped array ends) reads global
// memory instead.  Links have no reuse within a parity and stay plain loads.
// Blocks are ordered (site block, parity, rhs) with the rhs fastest, so the
// right-hand sides of one site block read the same links back to back (L2).
// ---------------------------------------------------------------------------
constexpr int TMA_TB = 128;                 // sites per block
constexpr long long TMA_SPIN = 1ll << 22;   // bounded mbarrier wait (polls; also 2 s of wall time)

struct TmaPlan {
    int cap[5];        // slots per range
    int spin_off[5];   // byte offsets of the spinor slots
    int nrm_off[5];    // byte offsets of the scale slots (16-bit storage)
    int bytes;         // dynamic shared memory
};

__host__ __device__ inline TmaPlan tma_plan(int Lxh, int nch, bool nrm)
{
    TmaPlan P;
    int off = 16;  // the mbarrier
    for (int j = 0; j < 5; ++j) {
        P.cap[j] = j == 0 ? TMA_TB + 2 * Lxh + 2 : TMA_TB;
        P.spin_off[j] = off;
        off += nch * P.cap[j] * 16;
    }
    for (int j = 0; j < 5; ++j) {
        P.nrm_off[j] = off;
        if (nrm) off += ((P.cap[j] + 8) * 4 + 15) & ~15;
    }
    P.bytes = off;
    return P;
}

__device__ __forceinline__ void tma_mbar_init(uint64_t* b)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tma_expect(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool tma_wait(uint64_t* b, long long polls)
{
    const unsigned long long t0 = global_ns();
    for (long long i = 0; i < polls; ++i) {
        if ((i & 1023) == 1023 && global_ns() - t0 > WAIT_LIMIT_NS) return false;
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(b))
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// spinor of slot i of a staged range (chunk-major, `cap` slots per chunk)
template <int SP>
__device__ __forceinline__ void load_spinor_smem(const uint8_t* base, const float* nrm, int cap, int i, float v[24])
{
    if constexpr (SP == P_F32) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(base + ((size_t)k * cap + i) * 16);
            v[4 * k] = a.x;
            v[4 * k + 1] = a.y;
            v[4 * k + 2] = a.z;
            v[4 * k + 3] = a.w;
        }
    } else {
        const float n = *nrm;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 a = *reinterpret_cast<const uint4*>(base + ((size_t)k * cap + i) * 16);
            const float2 a0 = Half<SP>::to2(a.x), a1 = Half<SP>::to2(a.y), a2 = Half<SP>::to2(a.z),
                         a3 = Half<SP>::to2(a.w);
            v[8 * k + 0] = a0.x * n;
            v[8 * k + 1] = a0.y * n;
            v[8 * k + 2] = a1.x * n;
            v[8 * k + 3] = a1.y * n;
            v[8 * k + 4] = a2.x * n;
            v[8 * k + 5] = a2.y * n;
            v[8 * k + 6] = a3.x * n;
            v[8 * k + 7] = a3.y * n;
        }
    }
}

struct TmaRange {
    int a, n, na;  // first staged index, count, first staged scale index
};

// lk: rows 0-1 of the hop's link, loaded before the wait (PRE), else loaded here
template <int SP, int GP, int MU, int S, bool PRE>
__device__ __forceinline__ void hop_tma(const DslashArgs& A, const uint8_t* sm, const TmaPlan& P, const TmaRange& rg,
                                        int j, const char* in_q, const float* inn_q, int p, int s, int sn, bool cross,
                                        const float* lk, float acc[24])
{
    float v[24];
    const int i = sn - rg.a;
    if ((unsigned)i < (unsigned)rg.n) {
        const float* nrm = nullptr;
        if constexpr (SP == P_F16 || SP == P_BF16)
            nrm = reinterpret_cast<const float*>(sm + P.nrm_off[j]) + (sn - rg.na);
        load_spinor_smem<SP>(sm + P.spin_off[j], nrm, P.cap[j], i, v);
    } else {
        load_spinor<SP, float>(in_q, inn_q, A.g.Vh, sn, v);
    }
    float h[12];
    project<MU, S, float>(v, h);
    if (cross) {
        const float ph = A.g.fbc[MU];
#pragma unroll
        for (int k = 0; k < 12; ++k) h[k] *= ph;
    }
    float u[18];
    if constexpr (PRE) {
#pragma unroll
        for (int k = 0; k < 12; ++k) u[k] = lk[k];
        link_row2<float>(u);
    } else {
        const int lpar = S > 0 ? p : 1 - p;
        const int ls = S > 0 ? s : sn;
        const char* lb = A.gauge + ((size_t)(lpar * 4 + MU) * A.g.Vh) * gauge_link_bytes_dev<GP>();
        load_link<GP, float>(lb, A.g.Vh, ls, u);
    }
    float chi[12];
    link_mul<S, float>(u, h, chi);
    accumulate<MU, S, float>(acc, chi);
}

template <int GP>
__device__ __forceinline__ void prefetch_link(const DslashArgs& A, int lpar, int mu, int ls, float w[12])
{
    const char* lb = A.gauge + ((size_t)(lpar * 4 + mu) * A.g.Vh) * gauge_link_bytes_dev<GP>();
    float u[18];
    load_link_rows<GP, float>(lb, A.g.Vh, ls, u);
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = u[k];
}

// PRE: every thread loads the rows of its eight links while the bulk copies are in flight
template <int SP, int GP, int NY, bool PRE>
__global__ void __launch_bounds__(TMA_TB, PRE ? 3 : 1) dslash_tma_kernel(DslashArgs A)
{
    extern __shared__ __align__(16) uint8_t sm[];  // bulk copies need 16-byte alignment
    constexpr int SCH = nchunk_dev<SP>();
    constexpr bool NRM = SP == P_F16 || SP == P_BF16;
    const Geom& g = A.g;
    const int r = blockIdx.x % A.nrhs;
    const int rest = blockIdx.x / A.nrhs;
    const int p = rest & 1, q = 1 - p;
    const int s0 = (rest >> 1) * TMA_TB;
    const char* in_q = A.in + ((size_t)r * 2 + q) * SCH * 16 * g.Vh;
    const float* inn_q = NRM ? A.in_n + ((size_t)r * 2 + q) * g.Vh : nullptr;
    const TmaPlan P = tma_plan(g.Lxh, SCH, NRM);
    const int PL = g.Lxh * g.L[1], VL = PL * g.L[2];
    const int lo[5] = {s0 - g.Lxh - 1, s0 + PL, s0 - PL, s0 + VL, s0 - VL};
    TmaRange rg[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int a = lo[j] < 0 ? 0 : lo[j];
        const int e = lo[j] + P.cap[j] > g.Vh ? g.Vh : lo[j] + P.cap[j];
        rg[j].a = a;
        rg[j].n = e > a ? e - a : 0;
        rg[j].na = a & ~3;
    }
    const int s = s0 + threadIdx.x;
    int c[4] = {0, 0, 0, 0};
    if (s < g.Vh) cb_coords(g, s, p, c);
    int nbr[8];
    cb_neighbours(g, s, c, nbr);
    // hops crossing the lattice boundary (they carry the boundary phase)
    const bool xp0 = c[0] + 1 == g.L[0], xm0 = c[0] == 0, yp0 = c[1] + 1 == g.L[1], ym0 = c[1] == 0;
    const bool zp0 = c[2] + 1 == g.L[2], zm0 = c[2] == 0, tp0 = c[3] + 1 == g.L[3], tm0 = c[3] == 0;
    const int* nb = nbr;
    float lk[PRE ? 8 : 1][12];
    if constexpr (PRE) {
        if (s < g.Vh) {
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int mu = h >> 1;
                const bool fwd = (h & 1) == 0;
                prefetch_link<GP>(A, fwd ? p : q, mu, fwd ? s : nb[h], lk[h]);
            }
        }
    }

    uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
    if (threadIdx.x == 0) tma_mbar_init(bar);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t total = 0;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            if (rg[j].n == 0) continue;
            total += SCH * rg[j].n * 16;
            if (NRM) total += ((((rg[j].a + rg[j].n + 3) & ~3) - rg[j].na) * 4);
        }
        tma_expect(bar, total);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            if (rg[j].n == 0) continue;
            for (int k = 0; k < SCH; ++k)
                bulk_g2s(sm + P.spin_off[j] + (size_t)k * P.cap[j] * 16, in_q + ((size_t)k * g.Vh + rg[j].a) * 16,
                         rg[j].n * 16, bar);
            if (NRM) {
                const int ne = (rg[j].a + rg[j].n + 3) & ~3;
                bulk_g2s(sm + P.nrm_off[j], inn_q + rg[j].na, (ne - rg[j].na) * 4, bar);
            }
        }
    }
    if (!tma_wait(bar, A.wait_polls)) {
        // the copies did not complete within the first wait's limit: report, drain them with a wait of the
        // full limit (no block exits with bulk copies in flight), write nothing
        if (A.err) atomicExch(A.err, 1u);
        tma_wait(bar, TMA_SPIN);
        return;
    }
    if (s >= g.Vh) return;

    float acc[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) acc[i] = 0.f;
    hop_tma<SP, GP, 0, +1, PRE>(A, sm, P, rg[0], 0, in_q, inn_q, p, s, nb[0], xp0, lk[0], acc);
    hop_tma<SP, GP, 0, -1, PRE>(A, sm, P, rg[0], 0, in_q, inn_q, p, s, nb[1], xm0, lk[PRE ? 1 : 0], acc);
    hop_tma<SP, GP, 1, +1, PRE>(A, sm, P, rg[0], 0, in_q, inn_q, p, s, nb[2], yp0, lk[PRE ? 2 : 0], acc);
    hop_tma<SP, GP, 1, -1, PRE>(A, sm, P, rg[0], 0, in_q, inn_q, p, s, nb[3], ym0, lk[PRE ? 3 : 0], acc);
    hop_tma<SP, GP, 2, +1, PRE>(A, sm, P, rg[1], 1, in_q, inn_q, p, s, nb[4], zp0, lk[PRE ? 4 : 0], acc);
    hop_tma<SP, GP, 2, -1, PRE>(A, sm, P, rg[2], 2, in_q, inn_q, p, s, nb[5], zm0, lk[PRE ? 5 : 0], acc);
    hop_tma<SP, GP, 3, +1, PRE>(A, sm, P, rg[3], 3, in_q, inn_q, p, s, nb[6], tp0, lk[PRE ? 6 : 0], acc);
    hop_tma<SP, GP, 3, -1, PRE>(A, sm, P, rg[4], 4, in_q, inn_q, p, s, nb[7], tm0, lk[PRE ? 7 : 0], acc);
    epilogue<SP, NY>(A, r, p, s, acc);
}

template <int SP, int GP, bool PRE>
cudaError_t launch_tma(const DslashArgs& A, int ny, cudaStream_t st)
{
    if constexpr (wide_dev<SP>) {
        return cudaErrorInvalidValue;
    } else {
        constexpr bool NRM = SP == P_F16 || SP == P_BF16;
        const TmaPlan P = tma_plan(A.g.Lxh, nchunk_dev<SP>(), NRM);
        if (P.bytes > 200 * 1024) return cudaErrorInvalidValue;
        static bool attr_set[4] = {false, false, false, false};
        if (!attr_set[ny]) {
            cudaError_t e = cudaSuccess;
            const int lim = 200 * 1024;
            switch (ny) {
            case 0: e = cudaFuncSetAttribute(dslash_tma_kernel<SP, GP, 0, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); break;
            case 1: e = cudaFuncSetAttribute(dslash_tma_kernel<SP, GP, 1, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); break;
            case 2: e = cudaFuncSetAttribute(dslash_tma_kernel<SP, GP, 2, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); break;
            case 3: e = cudaFuncSetAttribute(dslash_tma_kernel<SP, GP, 3, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); break;
            default: return cudaErrorInvalidValue;
            }
            if (e != cudaSuccess) return e;
            attr_set[ny] = true;
        }
        const long long nb = 2LL * ((A.g.Vh + TMA_TB - 1) / TMA_TB) * A.nrhs;
        if (nb > 0x7fffffffLL) return cudaErrorInvalidValue;
        const dim3 grid((unsigned)nb);
        switch (ny) {
        case 0: dslash_tma_kernel<SP, GP, 0, PRE><<<grid, TMA_TB, P.bytes, st>>>(A); break;
        case 1: dslash_tma_kernel<SP, GP, 1, PRE><<<grid, TMA_TB, P.bytes, st>>>(A); break;
        case 2: dslash_tma_kernel<SP, GP, 2, PRE><<<grid, TMA_TB, P.bytes, st>>>(A); break;
        case 3: dslash_tma_kernel<SP, GP, 3, PRE><<<grid, TMA_TB, P.bytes, st>>>(A); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
}

struct Staged {
    template <int SP, int GP>
    static cudaError_t run(const DslashArgs& A, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
    {
        switch (var) {
        case 3: return launch_staged<SP, GP>(A, ny, grid, block, st);
        case 4: return launch_tma<SP, GP, false>(A, ny, st);
        case 5: return launch_tma<SP, GP, true>(A, ny, st);
        }
        return cudaErrorInvalidValue;
    }
};

}  // namespace

cudaError_t launch_dslash_staged(const DslashArgs& A, int sp, int gp, int ny, int var, dim3 grid, dim3 block, cudaStream_t st)
{
    return dispatch_prec<Staged>(A, sp, gp, ny, var, grid, block, st);
}

}  // namespace ov
