// Layout conversion, level-1 vector kernels and deterministic FP64
// reductions on the internal even/odd layout.
//
// Reductions (global dots and norms, Sec. III: "scalar product and vector
// norm") accumulate in FP64 whatever the storage precision: each block
// reduces a fixed, grid-strided set of sites with warp shuffles and writes
// one partial per right-hand side; a second kernel sums the partials of each
// right-hand side in a fixed order, so results are bitwise reproducible.
#include <type_traits>

#include "ov_internal.cuh"
#include "ov_kernels.h"

namespace ov {

namespace {

constexpr int RB_THREADS = 256;

template <int P>
using creal_t = typename std::conditional<P == P_F64, double, typename std::conditional<P == P_DF64, df64, float>::type>::type;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of up to 2 doubles; result valid in thread 0
template <int NC>
__device__ __forceinline__ void block_sum(double v[NC])
{
    __shared__ double sh[NC][RB_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        double t = warp_sum(v[c]);
        if (lane == 0) sh[c][w] = t;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double t = lane < (int)(blockDim.x >> 5) ? sh[c][lane] : 0.0;
            v[c] = warp_sum(t);
        }
    }
}

// ------------------------------------------------------------------ pack / unpack
template <int P>
__global__ void pack_kernel(Geom g, const double2* __restrict__ canon, char* data, float* norm, int nrhs, int gamma5)
{
    const long V = 2L * g.Vh;
    const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (n >= V || r >= nrhs) return;
    const int x = (int)(n % g.L[0]);
    long rem = n / g.L[0];
    const int y = (int)(rem % g.L[1]);
    rem /= g.L[1];
    const int z = (int)(rem % g.L[2]);
    const int t = (int)(rem / g.L[2]);
    const int p = (x + y + z + t) & 1;
    const int s = (int)(n >> 1);
    using Real = creal_t<P>;
    Real v[24];
    const double2* src = canon + ((long)r * V + n) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 c = src[k];
        double sg = (gamma5 && k >= 6) ? -1.0 : 1.0;
        v[2 * k] = (Real)(sg * c.x);
        v[2 * k + 1] = (Real)(sg * c.y);
    }
    constexpr size_t CH = nchunk_dev<P>() * 16;
    const size_t off = ((size_t)r * 2 + p) * CH * g.Vh;
    store_spinor<P, Real>(data + off, norm ? norm + ((size_t)r * 2 + p) * g.Vh : nullptr, g.Vh, s, v);
}

template <int P>
__global__ void unpack_kernel(Geom g, const char* data, const float* norm, double2* canon, int nrhs, int gamma5)
{
    const long V = 2L * g.Vh;
    const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (n >= V || r >= nrhs) return;
    const int x = (int)(n % g.L[0]);
    long rem = n / g.L[0];
    const int y = (int)(rem % g.L[1]);
    rem /= g.L[1];
    const int z = (int)(rem % g.L[2]);
    const int t = (int)(rem / g.L[2]);
    const int p = (x + y + z + t) & 1;
    const int s = (int)(n >> 1);
    constexpr size_t CH = nchunk_dev<P>() * 16;
    const size_t off = ((size_t)r * 2 + p) * CH * g.Vh;
    double v[24];
    load_spinor<P, double>(data + off, norm ? norm + ((size_t)r * 2 + p) * g.Vh : nullptr, g.Vh, s, v);
    double2* dst = canon + ((long)r * V + n) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double sg = (gamma5 && k >= 6) ? -1.0 : 1.0;
        dst[k] = make_double2(sg * v[2 * k], sg * v[2 * k + 1]);
    }
}

// ------------------------------------------------------------------ gauge packing
__device__ __forceinline__ void atomic_max_pos(unsigned* a, float v) { atomicMax(a, __float_as_uint(fmaxf(v, 0.f))); }

template <int P>
__device__ __forceinline__ void store_link(char* base, int Vh, int s, const double u[18])
{
    if constexpr (P == P_DF64) {  // all three rows
        float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const df64 a(u[2 * k]), c(u[2 * k + 1]);
            b[(size_t)k * Vh + s] = make_float4(a.hi, a.lo, c.hi, c.lo);
        }
    } else if constexpr (P == P_F64) {
        double2* b = reinterpret_cast<double2*>(base);
#pragma unroll
        for (int k = 0; k < 9; ++k) b[(size_t)k * Vh + s] = make_double2(u[2 * k], u[2 * k + 1]);
    } else if constexpr (P == P_F32) {
        float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            b[(size_t)k * Vh + s] = make_float4((float)u[4 * k], (float)u[4 * k + 1], (float)u[4 * k + 2], (float)u[4 * k + 3]);
    } else {
        uint2* b = reinterpret_cast<uint2*>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint2 t;
            t.x = Half<P>::from2((float)u[4 * k], (float)u[4 * k + 1]);
            t.y = Half<P>::from2((float)u[4 * k + 2], (float)u[4 * k + 3]);
            b[(size_t)k * Vh + s] = t;
        }
    }
}

template <int P>
__global__ void pack_gauge_kernel(Geom g, const double2* __restrict__ canon, char* out, unsigned* err)
{
    const long V = 2L * g.Vh;
    const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= V) return;
    const int x = (int)(n % g.L[0]);
    long rem = n / g.L[0];
    const int y = (int)(rem % g.L[1]);
    rem /= g.L[1];
    const int z = (int)(rem % g.L[2]);
    const int t = (int)(rem / g.L[2]);
    const int p = (x + y + z + t) & 1;
    const int s = (int)(n >> 1);
    float e_unit = 0.f, e_row = 0.f;
    for (int mu = 0; mu < 4; ++mu) {
        const double2* u = canon + (n * 4 + mu) * 9;
        double2 m[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) m[k] = u[k];
        if (err) {
            // U U^dag = 1
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double re = 0, im = 0;
                    for (int k = 0; k < 3; ++k) {
                        double2 a = m[3 * i + k], b = m[3 * j + k];
                        re += a.x * b.x + a.y * b.y;
                        im += a.y * b.x - a.x * b.y;
                    }
                    e_unit = fmaxf(e_unit, (float)hypot(re - (i == j ? 1.0 : 0.0), im));
                }
            // row 2 = conj(row0 x row1)
            for (int j = 0; j < 3; ++j) {
                int a = (j + 1) % 3, b = (j + 2) % 3;
                double2 r0a = m[a], r0b = m[b], r1a = m[3 + a], r1b = m[3 + b];
                double re = (r0a.x * r1b.x - r0a.y * r1b.y) - (r0b.x * r1a.x - r0b.y * r1a.y);
                double im = (r0a.x * r1b.y + r0a.y * r1b.x) - (r0b.x * r1a.y + r0b.y * r1a.x);
                e_row = fmaxf(e_row, (float)hypot(m[6 + j].x - re, m[6 + j].y + im));
            }
        }
        double w[18];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            w[2 * k] = m[k].x;
            w[2 * k + 1] = m[k].y;
        }
        char* base = out + ((size_t)(p * 4 + mu) * g.Vh) * gauge_link_bytes_dev<P>();
        store_link<P>(base, g.Vh, s, w);
    }
    if (err) {
        atomic_max_pos(err, e_unit);
        atomic_max_pos(err + 1, e_row);
    }
}

// ------------------------------------------------------------------ conversion
template <int PI, int PO>
__global__ void convert_kernel(Geom g, const char* in, const float* in_n, char* out, float* out_n, int nrhs)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (idx >= 2 * g.Vh || r >= nrhs) return;
    const int p = idx >= g.Vh, s = idx - p * g.Vh;
    using Real = typename std::conditional<
        PI == P_F64 || PO == P_F64, double,
        typename std::conditional<PI == P_DF64 || PO == P_DF64, df64, float>::type>::type;
    Real v[24];
    constexpr size_t CI = nchunk_dev<PI>() * 16, CO = nchunk_dev<PO>() * 16;
    const size_t rp = (size_t)r * 2 + p;
    load_spinor<PI, Real>(in + rp * CI * g.Vh, in_n ? in_n + rp * g.Vh : nullptr, g.Vh, s, v);
    store_spinor<PO, Real>(out + rp * CO * g.Vh, out_n ? out_n + rp * g.Vh : nullptr, g.Vh, s, v);
}

// ------------------------------------------------------------------ lincomb (+ norm)
template <int P, int K>
__global__ void __launch_bounds__(RB_THREADS) lincomb_kernel(Geom g, LincombArgs A)
{
    using Real = creal_t<P>;
    constexpr size_t CH = nchunk_dev<P>() * 16;
    const int r = blockIdx.y;
    Real cre[K], cim[K];  // coefficients in the arithmetic type, converted once per thread
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const double2 cf = A.dcoef ? A.dcoef[j * A.out.nrhs + r] : A.hcoef[j];
        cre[j] = (Real)cf.x;
        cim[j] = (Real)cf.y;
    }
    double nrm = 0.0;
    const int N = 2 * g.Vh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        const int p = idx >= g.Vh, s = idx - p * g.Vh;
        const size_t rp = (size_t)r * 2 + p;
        Real o[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) o[i] = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            Real v[24];
            load_spinor<P, Real>(A.x[j].data + rp * CH * g.Vh, A.x[j].norm ? A.x[j].norm + rp * g.Vh : nullptr, g.Vh,
                                 s, v);
            const Real cr = cre[j], ci = cim[j];
            const bool g5 = (A.g5mask >> j) & 1;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                Real sg = (g5 && k >= 6) ? Real(-1) : Real(1);
                Real vr = sg * v[2 * k], vi = sg * v[2 * k + 1];
                o[2 * k] += cr * vr - ci * vi;
                o[2 * k + 1] += cr * vi + ci * vr;
            }
        }
        if (A.partials) {
            Real t = 0;
#pragma unroll
            for (int i = 0; i < 24; ++i) t += o[i] * o[i];
            nrm += (double)t;
        }
        store_spinor<P, Real>(A.out.data + rp * CH * g.Vh, A.out.norm ? A.out.norm + rp * g.Vh : nullptr, g.Vh, s, o);
    }
    if (A.partials) {
        double v[1] = {nrm};
        block_sum<1>(v);
        if (threadIdx.x == 0) A.partials[(size_t)r * gridDim.x + blockIdx.x] = v[0];
    }
}

// ------------------------------------------------------------------ dot
template <int P>
__global__ void __launch_bounds__(RB_THREADS) dot_kernel(Geom g, FieldDesc x, FieldDesc y, double2* partials)
{
    using Real = creal_t<P>;
    constexpr size_t CH = nchunk_dev<P>() * 16;
    const int r = blockIdx.y;
    double re = 0, im = 0;
    const int N = 2 * g.Vh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        const int p = idx >= g.Vh, s = idx - p * g.Vh;
        const size_t rp = (size_t)r * 2 + p;
        Real a[24], b[24];
        load_spinor<P, Real>(x.data + rp * CH * g.Vh, x.norm ? x.norm + rp * g.Vh : nullptr, g.Vh, s, a);
        load_spinor<P, Real>(y.data + rp * CH * g.Vh, y.norm ? y.norm + rp * g.Vh : nullptr, g.Vh, s, b);
        Real tr = 0, ti = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            tr += a[2 * k] * b[2 * k] + a[2 * k + 1] * b[2 * k + 1];
            ti += a[2 * k] * b[2 * k + 1] - a[2 * k + 1] * b[2 * k];
        }
        re += (double)tr;
        im += (double)ti;
    }
    double v[2] = {re, im};
    block_sum<2>(v);
    if (threadIdx.x == 0) partials[(size_t)r * gridDim.x + blockIdx.x] = make_double2(v[0], v[1]);
}

template <int NC>
__global__ void __launch_bounds__(RB_THREADS) finalize_kernel(const double* partials, int nblk, double* out)
{
    const int r = blockIdx.x;
    double v[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] += partials[((size_t)r * nblk + b) * NC + c];
    block_sum<NC>(v);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < NC; ++c) out[r * NC + c] = v[c];
}

// uniform(-1, 1) from a counter-based hash (splitmix64 of seed and element index)
__device__ __forceinline__ double hash_uniform(unsigned long long seed, unsigned long long i)
{
    unsigned long long z = seed * 0x9E3779B97F4A7C15ull + i + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

template <int P>
__global__ void fill_random_kernel(Geom g, FieldDesc f, unsigned long long seed)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (idx >= 2 * g.Vh) return;
    const int p = idx >= g.Vh, s = idx - p * g.Vh;
    double v[24];
    const unsigned long long base = ((unsigned long long)r * 2 * g.Vh + idx) * 24ull;
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = hash_uniform(seed, base + k);
    constexpr size_t CH = nchunk_dev<P>() * 16;
    const size_t rp = (size_t)r * 2 + p;
    store_spinor<P, double>(f.data + rp * CH * g.Vh, f.norm ? f.norm + rp * g.Vh : nullptr, g.Vh, s, v);
}

template <template <int> class F, typename... Args>
cudaError_t dispatch_prec(int prec, Args&&... args)
{
    switch (prec) {
    case P_F64: return F<P_F64>::run(args...);
    case P_F32: return F<P_F32>::run(args...);
    case P_F16: return F<P_F16>::run(args...);
    case P_BF16: return F<P_BF16>::run(args...);
    case P_DF64: return F<P_DF64>::run(args...);
    }
    return cudaErrorInvalidValue;
}

template <int P> struct PackRun {
    static cudaError_t run(const Geom& g, const double* canon, const FieldDesc& f, int gamma5, cudaStream_t st)
    {
        dim3 grid((unsigned)((2L * g.Vh + 127) / 128), f.nrhs);
        pack_kernel<P><<<grid, 128, 0, st>>>(g, (const double2*)canon, f.data, f.norm, f.nrhs, gamma5);
        return cudaGetLastError();
    }
};
template <int P> struct UnpackRun {
    static cudaError_t run(const Geom& g, const FieldDesc& f, double* canon, int gamma5, cudaStream_t st)
    {
        dim3 grid((unsigned)((2L * g.Vh + 127) / 128), f.nrhs);
        unpack_kernel<P><<<grid, 128, 0, st>>>(g, f.data, f.norm, (double2*)canon, f.nrhs, gamma5);
        return cudaGetLastError();
    }
};
template <int P> struct GaugeRun {
    static cudaError_t run(const Geom& g, const double* canon, void* out, unsigned* err, cudaStream_t st)
    {
        pack_gauge_kernel<P><<<(unsigned)((2L * g.Vh + 127) / 128), 128, 0, st>>>(g, (const double2*)canon,
                                                                                    (char*)out, err);
        return cudaGetLastError();
    }
};
template <int P> struct DotRun {
    static cudaError_t run(const Geom& g, const FieldDesc& x, const FieldDesc& y, double2* partials, int nblk,
                           cudaStream_t st)
    {
        dot_kernel<P><<<dim3(nblk, x.nrhs), RB_THREADS, 0, st>>>(g, x, y, partials);
        return cudaGetLastError();
    }
};
template <int P> struct LincombRun {
    static cudaError_t run(const Geom& g, const LincombArgs& A, int nblk, cudaStream_t st)
    {
        dim3 grid(nblk, A.out.nrhs);
        switch (A.K) {
        case 1: lincomb_kernel<P, 1><<<grid, RB_THREADS, 0, st>>>(g, A); break;
        case 2: lincomb_kernel<P, 2><<<grid, RB_THREADS, 0, st>>>(g, A); break;
        case 3: lincomb_kernel<P, 3><<<grid, RB_THREADS, 0, st>>>(g, A); break;
        case 4: lincomb_kernel<P, 4><<<grid, RB_THREADS, 0, st>>>(g, A); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
};

template <int P> struct FillRun {
    static cudaError_t run(const Geom& g, const FieldDesc& f, unsigned long long seed, cudaStream_t st)
    {
        fill_random_kernel<P><<<dim3((2 * g.Vh + 127) / 128, f.nrhs), 128, 0, st>>>(g, f, seed);
        return cudaGetLastError();
    }
};

template <int PI, int PO>
cudaError_t convert2(const Geom& g, const FieldDesc& in, const FieldDesc& out, cudaStream_t st)
{
    dim3 grid((2 * g.Vh + 127) / 128, in.nrhs);
    convert_kernel<PI, PO><<<grid, 128, 0, st>>>(g, in.data, in.norm, out.data, out.norm, in.nrhs);
    return cudaGetLastError();
}
template <int PI> struct ConvertRun {
    static cudaError_t run(const Geom& g, const FieldDesc& in, const FieldDesc& out, cudaStream_t st)
    {
        switch (out.prec) {
        case P_F64: return convert2<PI, P_F64>(g, in, out, st);
        case P_F32: return convert2<PI, P_F32>(g, in, out, st);
        case P_F16: return convert2<PI, P_F16>(g, in, out, st);
        case P_BF16: return convert2<PI, P_BF16>(g, in, out, st);
        case P_DF64: return convert2<PI, P_DF64>(g, in, out, st);
        }
        return cudaErrorInvalidValue;
    }
};

}  // namespace

int reduce_blocks(const Geom& g)
{
    int need = (2 * g.Vh + RB_THREADS - 1) / RB_THREADS;
    return need < 152 * 8 ? need : 152 * 8;
}

cudaError_t launch_pack(const Geom& g, const double* canon, const FieldDesc& f, int gamma5, cudaStream_t st)
{
    return dispatch_prec<PackRun>(f.prec, g, canon, f, gamma5, st);
}
cudaError_t launch_unpack(const Geom& g, const FieldDesc& f, double* canon, int gamma5, cudaStream_t st)
{
    return dispatch_prec<UnpackRun>(f.prec, g, f, canon, gamma5, st);
}
cudaError_t launch_pack_gauge(const Geom& g, const double* canon, void* out, int prec, unsigned* dev_err,
                              cudaStream_t st)
{
    return dispatch_prec<GaugeRun>(prec, g, canon, out, dev_err, st);
}
cudaError_t launch_convert(const Geom& g, const FieldDesc& in, const FieldDesc& out, cudaStream_t st)
{
    if (in.nrhs != out.nrhs) return cudaErrorInvalidValue;
    return dispatch_prec<ConvertRun>(in.prec, g, in, out, st);
}
cudaError_t launch_lincomb(const Geom& g, const LincombArgs& A, int nblk, cudaStream_t st)
{
    for (int j = 0; j < A.K; ++j)
        if (A.x[j].prec != A.out.prec || A.x[j].nrhs != A.out.nrhs) return cudaErrorInvalidValue;
    return dispatch_prec<LincombRun>(A.out.prec, g, A, nblk, st);
}
cudaError_t launch_dot(const Geom& g, const FieldDesc& x, const FieldDesc& y, double2* partials, int nblk,
                       cudaStream_t st)
{
    if (x.prec != y.prec || x.nrhs != y.nrhs) return cudaErrorInvalidValue;
    return dispatch_prec<DotRun>(x.prec, g, x, y, partials, nblk, st);
}
cudaError_t launch_fill_random(const Geom& g, const FieldDesc& f, unsigned long long seed, cudaStream_t st)
{
    return dispatch_prec<FillRun>(f.prec, g, f, seed, st);
}
cudaError_t launch_finalize(const double* partials, int nblk, int nrhs, int ncomp, double* out, cudaStream_t st)
{
    if (ncomp == 1)
        finalize_kernel<1><<<nrhs, RB_THREADS, 0, st>>>(partials, nblk, out);
    else
        finalize_kernel<2><<<nrhs, RB_THREADS, 0, st>>>(partials, nblk, out);
    return cudaGetLastError();
}

}  // namespace ov
