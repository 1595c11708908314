// Low-mode projection c = eta^dag psi (Eqs. 6-7, 9) on the 5th-generation
// tensor cores: the one dense contraction on the path.
//
// As a real GEMM: A = the eigenvectors, one row per eigenvector, each row the
// 24V reals of the field in the internal FP32 order (re, im interleaved),
// stored as bf16; B = two real columns per right-hand side, b1 = psi (re, im)
// and b2 = (im, -re), so that sum_k A_ik b1_k = Re(eta_i^dag psi) and
// sum_k A_ik b2_k = Im(eta_i^dag psi).  D[128 x N] = A[128 x K] B[K x N] is
// split over K across the CTAs: each CTA streams its K range through a
// 4-stage ring of shared-memory tiles filled by TMA (128B swizzle, K-major),
// one thread issues tcgen05.mma (kind::f16, bf16 in, FP32 accumulate in
// TMEM), the accumulator is read back with tcgen05.ld and written as FP32
// partial sums, and a second kernel adds the partials in a fixed order in
// FP64.  Rows beyond the number of eigenvectors and columns beyond 2R are
// zero-filled by the TMA bounds.
//
// Every wait on an mbarrier is bounded; on timeout the kernel records an
// error code, stops issuing work, waits (bounded) for its own copies and
// MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "ctx.h"

namespace ov {

namespace {

constexpr int TC_M = 128;         // rows of the MMA tile (eigenvectors per launch)
constexpr int TC_BK = 64;         // K elements per stage (128 bytes of bf16: one swizzle atom row)
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 128;
constexpr long long TC_SPIN = 1ll << 22;  // bounded wait (iterations of try_wait, ~seconds)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity)
{
    const unsigned long long t0 = global_ns();
    for (long long i = 0; i < TC_SPIN; ++i) {
        if (mbar_try(b, parity)) return true;
        if ((i & 1023) == 1023 && global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc(const void* p)
{
    const uint64_t addr = smem_u32(p);
    return ((addr >> 4) & 0x3FFFull)     // start address
           | (1ull << 16)                // leading byte offset (unused for swizzled K-major)
           | ((1024ull >> 4) << 32)      // stride byte offset: 8 rows x 128 bytes
           | (1ull << 46)                // descriptor version
           | (2ull << 61);               // 128-byte swizzle
}

// instruction descriptor: kind::f16, bf16 x bf16 -> f32, both K-major, M x N
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4)                     // D: f32
           | (1u << 7)                   // A: bf16
           | (1u << 10)                  // B: bf16
           | ((uint32_t)(N >> 3) << 17)  // N / 8
           | ((uint32_t)(M >> 4) << 24); // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// partials[blockIdx.x][row][col] (FP32), row < 128, col < npad; K range split evenly over the grid
// nsplit = 2: a second A operand (the bf16 remainder rows, tmAlo) accumulates into TMEM columns
// [npad, 2 npad); partials then hold [128][2 npad] per CTA
__global__ void __launch_bounds__(TC_THREADS, 1)
    proj_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAlo,
                   const __grid_constant__ CUtensorMap tmB, int ktiles, int npad, int nsplit, int tmem_cols,
                   float* __restrict__ partials, int* err)
{
    extern __shared__ uint8_t dyn_smem[];
    __shared__ __align__(8) uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    // 1024-byte aligned stage buffers (swizzle atoms)
    uint8_t* base = (uint8_t*)(((uintptr_t)dyn_smem + 1023) & ~(uintptr_t)1023);
    const int a_bytes = TC_M * TC_BK * 2;
    const int b_bytes = npad * TC_BK * 2;
    const int stage_bytes = nsplit * a_bytes + b_bytes;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = (ktiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per;
    const int nt = max(0, min(ktiles, t0 + per) - t0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    int issued = 0;  // tiles whose MMAs were issued (MMA thread)
    if (warp == 0 && lane == 0) {
        // producer: TMA loads into the stage ring
        for (int t = 0; t < nt; ++t) {
            const int s = t % TC_STAGES;
            const uint32_t ph = (t / TC_STAGES) & 1;
            if (t >= TC_STAGES && !mbar_wait(&empty_bar[s], ph ^ 1)) {
                atomicExch(err, 1);
                abort_flag = 1;
                break;
            }
            if (*(volatile int*)&abort_flag) break;
            uint8_t* sa = base + s * stage_bytes;
            mbar_expect_tx(&full_bar[s], stage_bytes);
            const int k = (t0 + t) * TC_BK;
            tma_load_2d(sa, &tmA, k, 0, &full_bar[s]);
            if (nsplit == 2) tma_load_2d(sa + a_bytes, &tmAlo, k, 0, &full_bar[s]);
            tma_load_2d(sa + nsplit * a_bytes, &tmB, k, 0, &full_bar[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc(TC_M, npad);
        for (int t = 0; t < nt; ++t) {
            const int s = t % TC_STAGES;
            const uint32_t ph = (t / TC_STAGES) & 1;
            if (!mbar_wait(&full_bar[s], ph)) {
                atomicExch(err, 2);
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint8_t* sa = base + s * stage_bytes;
            uint8_t* sb = sa + nsplit * a_bytes;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                mma_bf16(tmem, smem_desc(sa + kk * 32), smem_desc(sb + kk * 32), idesc, (t > 0 || kk > 0) ? 1u : 0u);
                if (nsplit == 2)
                    mma_bf16(tmem + (uint32_t)npad, smem_desc(sa + a_bytes + kk * 32), smem_desc(sb + kk * 32), idesc,
                             (t > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&empty_bar[s]);  // frees the stage when these MMAs have read it
            ++issued;
        }
        mma_commit(&done_bar);  // arrives when every issued MMA has completed
    }
    __syncthreads();
    // wait for the accumulator (bounded); with no tile the done barrier still completes (empty commit)
    bool ok = mbar_wait(&done_bar, 0);
    if (!ok && threadIdx.x == 0) atomicExch(err, 3);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int ncol = nsplit * npad;
    float* out = partials + (size_t)blockIdx.x * TC_M * ncol;
    const int row = warp * 32 + lane;
    for (int c0 = 0; c0 < ncol; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) out[(size_t)row * ncol + c0 + j] = (ok && issued >= 0 && nt > 0) ? v[j] : 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// c[i][r] = (sum_g P[g][i][2r], sum_g P[g][i][2r+1]) in FP64, fixed order.  nsplit = 2: the columns
// 2R + 2r, 2R + 2r + 1 hold the products with the bf16 remainder of psi, and the second accumulator
// (columns npad + ...) the products of the remainder rows of eta; the three leading terms are added
// (hi.hi + hi.lo + lo.hi; lo.lo is below the FP32 resolution)
__global__ void proj_tc_reduce(const float* partials, int ngrid, int npad, int nsplit, int nev, int nrhs, double2* c)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nev * nrhs) return;
    const int i = k / nrhs, r = k % nrhs;
    const int ncol = nsplit * npad;
    double re = 0, im = 0;
    for (int g = 0; g < ngrid; ++g) {
        const float* p = partials + ((size_t)g * TC_M + i) * ncol;
        re += p[2 * r];
        im += p[2 * r + 1];
        if (nsplit == 2) {
            re += (double)p[2 * nrhs + 2 * r] + (double)p[npad + 2 * r];
            im += (double)p[2 * nrhs + 2 * r + 1] + (double)p[npad + 2 * r + 1];
        }
    }
    c[k] = make_double2(re, im);
}

// B operand: rows 2r = psi_r, 2r+1 = (im, -re) pairs, bf16, from an FP32 field; nsplit = 2 adds rows
// 2R + 2r, 2R + 2r + 1 with the bf16 remainders x - bf16(x) of the same values
__device__ __forceinline__ float bf16_rem(float x) { return x - __bfloat162float(__float2bfloat16_rn(x)); }
__global__ void build_b_kernel(const float4* __restrict__ x, int n4, int nrhs, int nsplit, __nv_bfloat16* B,
                               long long K)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (q >= n4 || r >= nrhs) return;
    const float4 v = x[(size_t)r * n4 + q];
    __nv_bfloat162* b1 = reinterpret_cast<__nv_bfloat162*>(B + (size_t)(2 * r) * K + 4 * q);
    __nv_bfloat162* b2 = reinterpret_cast<__nv_bfloat162*>(B + (size_t)(2 * r + 1) * K + 4 * q);
    b1[0] = __floats2bfloat162_rn(v.x, v.y);
    b1[1] = __floats2bfloat162_rn(v.z, v.w);
    b2[0] = __floats2bfloat162_rn(v.y, -v.x);
    b2[1] = __floats2bfloat162_rn(v.w, -v.z);
    if (nsplit == 2) {
        __nv_bfloat162* l1 = reinterpret_cast<__nv_bfloat162*>(B + (size_t)(2 * nrhs + 2 * r) * K + 4 * q);
        __nv_bfloat162* l2 = reinterpret_cast<__nv_bfloat162*>(B + (size_t)(2 * nrhs + 2 * r + 1) * K + 4 * q);
        l1[0] = __floats2bfloat162_rn(bf16_rem(v.x), bf16_rem(v.y));
        l1[1] = __floats2bfloat162_rn(bf16_rem(v.z), bf16_rem(v.w));
        l2[0] = __floats2bfloat162_rn(bf16_rem(v.y), bf16_rem(-v.x));
        l2[1] = __floats2bfloat162_rn(bf16_rem(v.w), bf16_rem(-v.z));
    }
}

// the bf16 remainder x - bf16(x) of each FP32 value
__global__ void to_bf16_lo_kernel(const float4* __restrict__ x, long long n4, __nv_bfloat16* y)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n4) return;
    const float4 v = x[q];
    const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) y[4 * q + j] = __float2bfloat16_rn(e[j] - __bfloat162float(__float2bfloat16_rn(e[j])));
}

__global__ void to_bf16_kernel(const float4* __restrict__ x, long long n4, __nv_bfloat16* y)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n4) return;
    const float4 v = x[q];
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(y + 4 * q);
    o[0] = __floats2bfloat162_rn(v.x, v.y);
    o[1] = __floats2bfloat162_rn(v.z, v.w);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2D bf16 map: rows x K (K contiguous), box 64 x box_rows, 128B swizzle, zero fill outside
bool make_map(CUtensorMap* m, const void* ptr, long long K, int rows, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// V c on the tensor cores (Eq. 7: psi_h = psi - sum_i eta_i c_i and the exact low-mode
// part sum_i sign(lam_i) c_i eta_i).  As a real GEMM over the eigenvector index i:
//   P[k][col] = sum_i eta_i[k] B[i][col],  k = a real position of the field (FP32 internal order),
// with four B columns per right-hand side r, (c_re, c_im, s c_re, s c_im) (s = sign(lam_i)), each
// split into a bf16 high part and a bf16 remainder (8 columns), so the coefficients lose nothing.
// Real position k = 2m holds Re eta(m), k = 2m + 1 holds Im eta(m); the complex product is
// assembled in the epilogue from the row and its neighbour (TMEM lanes k and k ^ 1):
//   corr_re(m) = X(2m) - Y(2m+1),  corr_im(m) = Y(2m) + X(2m+1),  X = P[.][c_re], Y = P[.][c_im].
// A = the eigenvector rows (bf16, [nev][48 Vh]) read as an MN-major operand: a tile is 128
// consecutive real positions (two 64-element swizzle atoms, LBO apart) by the eigenvector index
// (8-row groups 1024 bytes apart), loaded by TMA straight from the row-major copy; rows i >= nev
// are zero-filled by the TMA bounds and cost no traffic.  nsplit = 2 adds the rows of the bf16
// remainder eta - bf16(eta) into the same accumulator (FP32-class eigenvectors at 4 bytes per real).
// Persistent, warp-specialised: warp 0 issues the TMA loads into a ring of stages, warp 1 issues
// tcgen05.mma into one of two TMEM accumulators, warps 2-5 (one per TMEM lane quarter) drain the
// other accumulator and write the outputs, so loads, MMAs and stores overlap.
constexpr int UP_M = 128;
constexpr int UP_THREADS = 192;

struct UpArgs {
    long long ntiles;      // 48 Vh / 128
    int kpadA;             // A box rows: nev rounded up to 16
    int kchunksB;          // 64-element K chunks of B
    int npad;              // B rows = accumulator columns (8 per rhs, padded to 16)
    int nsplit;            // 1: eta rows; 2: also the remainder rows
    int stages;
    int R;
    int Vh;
    int mode;              // 0: FP32 fields, out1 = psi - corr, out2 = gamma5 w; 1: out1 = corr, out2 = gamma5 w
    const float* psi;      // FP32 field (mode 0)
    float* out1;
    float* out2;           // may be null
    int* err;
};

// MN-major operand descriptor, 128-byte swizzle: atoms of 64 MN elements x 8 K rows (1024 bytes),
// K groups SBO = 1024 bytes apart, the second MN atom LBO bytes further
__device__ __forceinline__ uint64_t smem_desc_mn(const void* p, uint32_t lbo)
{
    const uint64_t addr = smem_u32(p);
    return ((addr >> 4) & 0x3FFFull) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) | ((1024ull >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

__global__ void __launch_bounds__(UP_THREADS, 1)
    proj_update_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAlo,
                          const __grid_constant__ CUtensorMap tmB, UpArgs P)
{
    extern __shared__ uint8_t dyn_smem[];
    __shared__ __align__(8) uint64_t full_bar[4], empty_bar[4], tfull[2], tempty[2], bbar, fin_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ long long consumed;  // tiles whose stage the MMA thread has taken (for the producer's drain)
    uint8_t* base = (uint8_t*)(((uintptr_t)dyn_smem + 1023) & ~(uintptr_t)1023);
    const int S = P.stages;
    const uint32_t half_bytes = (uint32_t)P.kpadA * 128;             // one MN atom column of A
    const uint32_t stage_bytes = (uint32_t)P.nsplit * 2 * half_bytes;
    uint8_t* bsm = base + (size_t)S * stage_bytes;
    const uint32_t bchunk = (uint32_t)P.npad * 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncols = 2 * P.npad;
    const int tcols = ncols <= 32 ? 32 : (ncols <= 64 ? 64 : (ncols <= 128 ? 128 : 256));

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 4);
        }
        mbar_init(&bbar, 1);
        mbar_init(&fin_bar, 1);
        abort_flag = 0;
        consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const long long my_tiles = P.ntiles > blockIdx.x ? (P.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 0 && lane == 0) {
        // producer: B once, then the A tiles through the ring
        mbar_expect_tx(&bbar, (uint32_t)P.kchunksB * bchunk);
        for (int c = 0; c < P.kchunksB; ++c) tma_load_2d(bsm + (size_t)c * bchunk, &tmB, c * 64, 0, &bbar);
        long long it = 0;
        for (; it < my_tiles; ++it) {
            const int s = (int)(it % S);
            const uint32_t ph = (uint32_t)((it / S) & 1);
            if (it >= S && !mbar_wait(&empty_bar[s], ph ^ 1)) {
                atomicExch(P.err, 11);
                abort_flag = 1;
                break;
            }
            if (*(volatile int*)&abort_flag) break;
            const long long tile = blockIdx.x + it * gridDim.x;
            uint8_t* st = base + (size_t)s * stage_bytes;
            mbar_expect_tx(&full_bar[s], stage_bytes);
            const int x0 = (int)(tile * UP_M);
            tma_load_2d(st, &tmA, x0, 0, &full_bar[s]);
            tma_load_2d(st + half_bytes, &tmA, x0 + 64, 0, &full_bar[s]);
            if (P.nsplit == 2) {
                tma_load_2d(st + 2 * half_bytes, &tmAlo, x0, 0, &full_bar[s]);
                tma_load_2d(st + 3 * half_bytes, &tmAlo, x0 + 64, 0, &full_bar[s]);
            }
        }
        // drain: no block leaves with bulk copies in flight (the bounded waits of the stages that were
        // issued and never taken by the MMA thread)
        __threadfence_block();
        for (long long t = *(volatile long long*)&consumed; t < it; ++t)
            mbar_wait(&full_bar[t % S], (uint32_t)((t / S) & 1));
        mbar_wait(&bbar, 0);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc(UP_M, P.npad) | (1u << 15);  // A MN-major
        const int ksteps = P.kpadA / 16;
        bool ok = mbar_wait(&bbar, 0);
        if (!ok) {
            atomicExch(P.err, 12);
            abort_flag = 1;
        }
        for (long long it = 0; ok && it < my_tiles; ++it) {
            const int s = (int)(it % S);
            const int a = (int)(it & 1);
            if (*(volatile int*)&abort_flag) break;
            if (!mbar_wait(&full_bar[s], (uint32_t)((it / S) & 1))) {
                atomicExch(P.err, 13);
                abort_flag = 1;
                break;
            }
            consumed = it + 1;
            if (it >= 2 && !mbar_wait(&tempty[a], (uint32_t)(((it >> 1) & 1) ^ 1))) {
                atomicExch(P.err, 14);
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint8_t* st = base + (size_t)s * stage_bytes;
            const uint32_t d = tmem + (uint32_t)(a * P.npad);
            for (int sp = 0; sp < P.nsplit; ++sp)
                for (int j = 0; j < ksteps; ++j) {
                    const uint64_t ad = smem_desc_mn(st + (size_t)sp * 2 * half_bytes + (size_t)j * 2048, half_bytes);
                    const uint64_t bd = smem_desc(bsm + (size_t)(j >> 2) * bchunk + (j & 3) * 32);
                    mma_bf16(d, ad, bd, idesc, (sp > 0 || j > 0) ? 1u : 0u);
                }
            mma_commit(&empty_bar[s]);  // the stage is free once these MMAs have read it
            mma_commit(&tfull[a]);      // the accumulator is ready for the epilogue
        }
        mma_commit(&fin_bar);  // arrives when every MMA issued by this thread has completed
        if (!mbar_wait(&fin_bar, 0)) atomicExch(P.err, 15);
    } else if (warp >= 2) {
        // epilogue: TMEM lane quarter q of the accumulator, row = q * 32 + lane
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const long long rhs_reals = 48LL * P.Vh;
        const long long par_reals = 24LL * P.Vh;
        const long long lo_chunk = 12LL * P.Vh;  // chunks 3..5 of a parity (spins 2, 3) start here
        for (long long it = 0; it < my_tiles; ++it) {
            const int a = (int)(it & 1);
            if (*(volatile int*)&abort_flag) break;
            if (!mbar_wait(&tfull[a], (uint32_t)((it >> 1) & 1))) {
                if (lane == 0) atomicExch(P.err, 16);
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const long long tile = blockIdx.x + it * gridDim.x;
            const long long k = tile * UP_M + row;
            const bool lower = (k % par_reals) >= lo_chunk;  // gamma5 = -1 on spins 2, 3
            const float g5 = lower ? -1.f : 1.f;
            const float sg = (lane & 1) ? 1.f : -1.f;
            for (int c0 = 0; c0 < P.npad; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * P.npad + c0), v);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = (c0 >> 3) + h;  // 8 columns per rhs
                    const float X = v[8 * h + 0] + v[8 * h + 4], Y = v[8 * h + 1] + v[8 * h + 5];
                    const float XW = v[8 * h + 2] + v[8 * h + 6], YW = v[8 * h + 3] + v[8 * h + 7];
                    const float Yp = __shfl_xor_sync(0xffffffffu, Y, 1);
                    const float YWp = __shfl_xor_sync(0xffffffffu, YW, 1);
                    if (r < P.R) {
                        const float corr = X + sg * Yp, w = XW + sg * YWp;
                        const long long idx = (long long)r * rhs_reals + k;
                        P.out1[idx] = P.mode == 0 ? P.psi[idx] - corr : corr;
                        if (P.out2) P.out2[idx] = g5 * w;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[a])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// B[n][k] (bf16, [npad][kchunks * 64]): n = 8 r + j, k = eigenvector index; j = 0..3: high parts of
// (c_re, c_im, s c_re, s c_im), j = 4..7: their bf16 remainders; zero outside (r < R, k < nev)
__global__ void build_coef_b_kernel(const double2* __restrict__ cf, const double* __restrict__ sg, int nev, int R,
                                    int npad, int kp, __nv_bfloat16* B)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (k >= kp || n >= npad) return;
    float v = 0.f;
    const int r = n >> 3, j = n & 7;
    if (r < R && k < nev) {
        const double2 c = cf[(size_t)k * R + r];
        const double s = sg ? sg[k] : 0.0;
        const int t = j & 3;
        const double x = t == 0 ? c.x : (t == 1 ? c.y : (t == 2 ? s * c.x : s * c.y));
        const float hi = __bfloat162float(__float2bfloat16_rn((float)x));
        v = j < 4 ? hi : (float)(x - (double)hi);
    }
    B[(size_t)n * kp + k] = __float2bfloat16_rn(v);
}

// out1 = psi - corr and out2 = w (already gamma5-signed), corr and w FP32 fields, psi and the
// outputs in a 16-bit storage precision (per-site scale recomputed on store)
template <int P>
__global__ void proj_combine_kernel(Geom g, FieldDesc psi, const float* corr, const float* w, FieldDesc out1,
                                    FieldDesc out2)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (idx >= 2 * g.Vh) return;
    const int p = idx >= g.Vh, s = idx - p * g.Vh;
    const size_t rp = (size_t)r * 2 + p;
    constexpr size_t CH = nchunk_dev<P>() * 16;
    float a[24], c[24];
    load_spinor<P, float>(psi.data + rp * CH * g.Vh, psi.norm ? psi.norm + rp * g.Vh : nullptr, g.Vh, s, a);
    load_spinor<P_F32, float>(reinterpret_cast<const char*>(corr) + rp * 96 * g.Vh, nullptr, g.Vh, s, c);
#pragma unroll
    for (int i = 0; i < 24; ++i) a[i] -= c[i];
    store_spinor<P, float>(out1.data + rp * CH * g.Vh, out1.norm ? out1.norm + rp * g.Vh : nullptr, g.Vh, s, a);
    if (w) {
        load_spinor<P_F32, float>(reinterpret_cast<const char*>(w) + rp * 96 * g.Vh, nullptr, g.Vh, s, c);
        store_spinor<P, float>(out2.data + rp * CH * g.Vh, out2.norm ? out2.norm + rp * g.Vh : nullptr, g.Vh, s, c);
    }
}

}  // namespace

// bf16 copy of the eigenvectors (rows of A), built once from the FP32 copy
int eig_bf16_rows(ov_ctx* c, int which, cudaStream_t st, const void** out)
{
    EigSet& E = c->eig[which];
    if (!E.nev) return set_err(c, OV_ESTATE, "no eigenpairs stored (which=%d)", which);
    if (!E.tc_rows) {
        FieldDesc f32;
        OV_TRY(eig_vectors(c, which, P_F32, st, &f32));
        const long long K = 48LL * c->g.Vh;
        OV_TRY(dev_alloc(c, &E.tc_rows, (size_t)E.nev * K * 2));
        E.tc_bytes = (size_t)E.nev * K * 2;
        const long long n4 = (long long)E.nev * K / 4;
        to_bf16_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>((const float4*)f32.data, n4,
                                                                     (__nv_bfloat16*)E.tc_rows);
        OV_CUDA(c, cudaGetLastError());
    }
    *out = E.tc_rows;
    return OV_OK;
}

int eig_bf16_lo_rows(ov_ctx* c, int which, cudaStream_t st, const void** out)
{
    EigSet& E = c->eig[which];
    const void* hi = nullptr;
    OV_TRY(eig_bf16_rows(c, which, st, &hi));
    if (!E.tc_lo) {
        FieldDesc f32;
        OV_TRY(eig_vectors(c, which, P_F32, st, &f32));
        const long long K = 48LL * c->g.Vh;
        OV_TRY(dev_alloc(c, &E.tc_lo, (size_t)E.nev * K * 2));
        E.tc_lo_bytes = (size_t)E.nev * K * 2;
        // remainder of the FP32 copy: hi + lo carries 16 significand bits of the FP32 value, which is what
        // the FP32 arithmetic of the operator resolves
        const long long n4 = (long long)E.nev * K / 4;
        to_bf16_lo_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>((const float4*)f32.data, n4,
                                                                        (__nv_bfloat16*)E.tc_lo);
        OV_CUDA(c, cudaGetLastError());
    }
    *out = E.tc_lo;
    return OV_OK;
}

// out1_r = psi_r - sum_i eta_i c[i][r], out2_r = gamma5 sum_i s_i c[i][r] eta_i (out2.data may be null)
// on the tensor cores; c: device double2 [nev][R], s: device sign(lam_i) (may be null).  16-bit
// storage reads the bf16 rows; FP32 storage adds the bf16 remainder rows.
int proj_update_tc(ov_ctx* c, int which, const FieldDesc& psi, const double2* dcoef, const double* dsign,
                   const FieldDesc& out1, const FieldDesc& out2, cudaStream_t st)
{
    EigSet& E = c->eig[which];
    const int nev = E.nev, R = psi.nrhs;
    if (nev < 1 || nev > 128 || R > 16 || c->g.Vh % 8)
        return set_err(c, OV_EINVAL, "tensor-core update: nev %d (1..128), nrhs %d (<= 16), Vh %% 8", nev, R);
    const int P = psi.prec;
    if (P != P_F32 && P != P_F16 && P != P_BF16)
        return set_err(c, OV_EINVAL, "tensor-core update: FP32 or 16-bit storage only");
    const int nsplit = P == P_F32 ? 2 : 1;
    const void* A = nullptr;
    const void* Alo = nullptr;
    OV_TRY(eig_bf16_rows(c, which, st, &A));
    if (nsplit == 2) OV_TRY(eig_bf16_lo_rows(c, which, st, &Alo));
    const long long K = 48LL * c->g.Vh;
    const int npad = ((8 * R + 15) / 16) * 16;
    const int kpadA = ((nev + 15) / 16) * 16;
    const int kchunksB = (nev + 63) / 64;
    const int kpB = kchunksB * 64;
    const size_t bbytes_g = (size_t)npad * kpB * 2;
    if (c->tc_cb_bytes < bbytes_g) {
        if (c->tc_cb) {
            cudaDeviceSynchronize();
            dev_free(c, c->tc_cb, c->tc_cb_bytes);
        }
        c->tc_cb = nullptr;
        c->tc_cb_bytes = 0;
        graphs_clear(c);
        OV_TRY(dev_alloc(c, &c->tc_cb, bbytes_g));
        c->tc_cb_bytes = bbytes_g;
    }
    build_coef_b_kernel<<<dim3((kpB + 127) / 128, npad), 128, 0, st>>>(dcoef, out2.data ? dsign : nullptr, nev, R,
                                                                        npad, kpB, (__nv_bfloat16*)c->tc_cb);
    OV_CUDA(c, cudaGetLastError());
    CUtensorMap ma, malo, mb;
    if (!make_map(&ma, A, K, nev, kpadA) || !make_map(&malo, nsplit == 2 ? Alo : A, K, nev, kpadA) ||
        !make_map(&mb, c->tc_cb, kpB, npad, npad))
        return set_err(c, OV_ECUDA, "cuTensorMapEncodeTiled failed");
    const uint32_t stage_bytes = (uint32_t)nsplit * 2 * kpadA * 128;
    const uint32_t bbytes = (uint32_t)kchunksB * npad * 128;
    constexpr int kSmemMax = 224 * 1024;  // dynamic part; the barriers' static shared memory comes on top
    const int stages = std::min(4, (int)((kSmemMax - 1024 - (int)bbytes) / (int)stage_bytes));
    if (stages < 2) return set_err(c, OV_EINVAL, "tensor-core update: tiles do not fit in shared memory");
    const size_t smem = (size_t)stages * stage_bytes + bbytes + 1024;
    static const cudaError_t attr =
        cudaFuncSetAttribute(proj_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    OV_CUDA(c, attr);
    if (!c->tc_err) {
        void* p = nullptr;
        OV_TRY(dev_alloc(c, &p, sizeof(int)));
        c->tc_err = (int*)p;
        OV_CUDA(c, cudaMemsetAsync(c->tc_err, 0, sizeof(int), st));
    }
    UpArgs a;
    memset(&a, 0, sizeof a);
    a.ntiles = K / UP_M;
    a.kpadA = kpadA;
    a.kchunksB = kchunksB;
    a.npad = npad;
    a.nsplit = nsplit;
    a.stages = stages;
    a.R = R;
    a.Vh = c->g.Vh;
    a.err = c->tc_err;
    FieldDesc corr{}, wf{};
    if (P == P_F32) {
        a.mode = 0;
        a.psi = (const float*)psi.data;
        a.out1 = (float*)out1.data;
        a.out2 = out2.data ? (float*)out2.data : nullptr;
    } else {
        OV_TRY(ws_field(c, WS_TC0, P_F32, R, &corr));
        if (out2.data) OV_TRY(ws_field(c, WS_TC1, P_F32, R, &wf));
        a.mode = 1;
        a.out1 = (float*)corr.data;
        a.out2 = out2.data ? (float*)wf.data : nullptr;
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int grid = (int)std::min<long long>(a.ntiles, sms);
    proj_update_tc_kernel<<<grid, UP_THREADS, smem, st>>>(ma, malo, mb, a);
    OV_CUDA(c, cudaGetLastError());
    if (P != P_F32) {
        const dim3 g2((2 * c->g.Vh + 127) / 128, R);
        if (P == P_F16)
            proj_combine_kernel<P_F16><<<g2, 128, 0, st>>>(c->g, psi, (const float*)corr.data,
                                                           out2.data ? (const float*)wf.data : nullptr, out1, out2);
        else
            proj_combine_kernel<P_BF16><<<g2, 128, 0, st>>>(c->g, psi, (const float*)corr.data,
                                                            out2.data ? (const float*)wf.data : nullptr, out1, out2);
        OV_CUDA(c, cudaGetLastError());
    }
    return OV_OK;
}

// c[i][r] = eta_i^dag psi_r (double2 [nev][R] device) on the tensor cores; psi any precision
int proj_dots_tc(ov_ctx* c, int which, const FieldDesc& psi, double2* cout, cudaStream_t st, int nsplit)
{
    EigSet& E = c->eig[which];
    const int nev = E.nev, R = psi.nrhs;
    if (nev < 1 || nev > TC_M) return set_err(c, OV_EINVAL, "tensor-core projection: nev = %d outside 1..128", nev);
    if (nsplit != 1 && nsplit != 2) return set_err(c, OV_EINVAL, "tensor-core projection: nsplit %d", nsplit);
    const int ncolB = 2 * nsplit * R;  // B rows: (psi, i psi) per rhs, and their bf16 remainders
    const int npad = ((ncolB + 15) / 16) * 16;
    if (npad * nsplit > 256) return set_err(c, OV_EINVAL, "tensor-core projection: too many right-hand sides");
    const long long K = 48LL * c->g.Vh;
    if (K % TC_BK) return set_err(c, OV_EINVAL, "tensor-core projection: 24V must be a multiple of 64");
    const void* A = nullptr;
    const void* Alo = nullptr;
    OV_TRY(eig_bf16_rows(c, which, st, &A));
    if (nsplit == 2) OV_TRY(eig_bf16_lo_rows(c, which, st, &Alo));
    // psi as FP32 (internal order), then the bf16 B rows
    FieldDesc p32 = psi;
    if (psi.prec != P_F32) {
        OV_TRY(ws_field(c, WS_AUX0, P_F32, R, &p32));
        OV_TRY(convert(c, psi, p32, st));
    }
    const size_t bbytes = (size_t)ncolB * K * 2;
    if (c->tc_b_bytes < bbytes) {
        if (c->tc_b) {
            cudaDeviceSynchronize();
            dev_free(c, c->tc_b, c->tc_b_bytes);
        }
        c->tc_b = nullptr;
        c->tc_b_bytes = 0;
        graphs_clear(c);
        OV_TRY(dev_alloc(c, &c->tc_b, bbytes));
        c->tc_b_bytes = bbytes;
    }
    const long long n4 = K / 4;
    build_b_kernel<<<dim3((unsigned)((n4 + 255) / 256), R), 256, 0, st>>>((const float4*)p32.data, (int)n4, R, nsplit,
                                                                           (__nv_bfloat16*)c->tc_b, K);
    OV_CUDA(c, cudaGetLastError());
    CUtensorMap ma, malo, mb;
    if (!make_map(&ma, A, K, nev, TC_M) || !make_map(&malo, nsplit == 2 ? Alo : A, K, nev, TC_M) ||
        !make_map(&mb, c->tc_b, K, ncolB, npad))
        return set_err(c, OV_ECUDA, "cuTensorMapEncodeTiled failed");
    const int ktiles = (int)(K / TC_BK);
    const int grid = std::min(ktiles, 2 * 152);
    const size_t smem = (size_t)TC_STAGES * (nsplit * TC_M + npad) * TC_BK * 2 + 1024;
    OV_TRY(ensure_partials(c, (size_t)grid * TC_M * nsplit * npad * sizeof(float)));
    if (!c->tc_err) {
        void* p = nullptr;
        OV_TRY(dev_alloc(c, &p, sizeof(int)));
        c->tc_err = (int*)p;
        OV_CUDA(c, cudaMemsetAsync(c->tc_err, 0, sizeof(int), st));
    }
    // once per process, for the largest ring: no attribute call inside a graph capture
    static const cudaError_t attr = cudaFuncSetAttribute(proj_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         TC_STAGES * (TC_M + 256) * TC_BK * 2 + 1024);
    OV_CUDA(c, attr);
    if (smem > (size_t)(TC_STAGES * (TC_M + 256) * TC_BK * 2 + 1024))
        return set_err(c, OV_EINVAL, "tensor-core projection: tiles do not fit in shared memory");
    const int ncol = nsplit * npad;
    const int tmem_cols = ncol <= 32 ? 32 : (ncol <= 64 ? 64 : (ncol <= 128 ? 128 : 256));
    proj_tc_kernel<<<grid, TC_THREADS, smem, st>>>(ma, malo, mb, ktiles, npad, nsplit, tmem_cols,
                                                   (float*)c->partials, c->tc_err);
    OV_CUDA(c, cudaGetLastError());
    proj_tc_reduce<<<(nev * R + 127) / 128, 128, 0, st>>>((const float*)c->partials, grid, npad, nsplit, nev, R,
                                                          cout);
    OV_CUDA(c, cudaGetLastError());
    return OV_OK;
}

int proj_tc_status(ov_ctx* c, cudaStream_t st)
{
    if (!c->tc_err) return OV_OK;
    int h = 0;
    OV_CUDA(c, cudaMemcpyAsync(&h, c->tc_err, sizeof h, cudaMemcpyDeviceToHost, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    if (h) {
        cudaMemsetAsync(c->tc_err, 0, sizeof(int), st);
        return set_err(c, OV_ETIMEOUT, "tensor-core projection: bounded wait gave up (stage %d)", h);
    }
    return OV_OK;
}

}  // namespace ov
