// Internal definitions of the GB300 overlap-fermion library: lattice
// geometry, the even/odd storage formats and their load/store routines.
//
// Canonical (user-facing) layout: complex128 [rhs][t][z][y][x][spin 4][colour 3],
// gauge complex128 [t][z][y][x][mu 4][3][3], mu = 0..3 <-> x, y, z, t.
//
// Internal layout (library-owned).  Sites are split by parity
// p = (x+y+z+t) & 1 and numbered within a parity by the checkerboard index
// s = (((t*Lz + z)*Ly + y)*Lx + x) / 2 (Lx even).  A spinor field of R
// right-hand sides is an array of 16-byte chunks
//     chunk[r][p][k][s],  k = 0 .. NCH-1,
// so a warp reading chunk k of 32 consecutive sites issues one coalesced
// 512-byte transaction.  The 24 reals of a site are ordered
// (spin, colour, re/im) and packed as 12 double2 (FP64), 6 float4 (FP32) or
// 3 x 8 16-bit values (FP16 / BF16) with one FP32 scale per site
// (norm[r][p][s] = max |component|, values stored divided by it).
// Gauge links: forward links only; FP32 and 16-bit keep only rows 0 and 1 of
// each SU(3) matrix (reconstruct-12): link[p][mu][k][s] = U_mu(n), n = site (p, s); chunks
// are 3 float4 (FP32) or 3 x 4 16-bit values; FP64 and double-float keep all
// three rows, 9 double2 (FP64) or 9 float4 (hi, lo, hi, lo).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include <string>

namespace ov {

// P_DF64: FP64-class "double-float" format: every real is an unevaluated sum
// hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2, about 48 significand bits),
// 8 bytes per real like FP64, computed on the FP32 pipes with error-free
// transformations.  GB300's FP64 units are a small fraction of its FP32
// throughput, so this is the fast form of the FP64-accurate operator.
enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_BF16 = 3, P_DF64 = 4 };
constexpr int NPREC = 5;

inline bool wide(int prec) { return prec == P_F64 || prec == P_DF64; }
inline int spinor_chunks(int prec) { return wide(prec) ? 12 : (prec == P_F32 ? 6 : 3); }
inline bool has_norm(int prec) { return prec == P_F16 || prec == P_BF16; }
inline size_t spinor_site_bytes(int prec) { return (size_t)spinor_chunks(prec) * 16; }
// links: reconstruct-12 (rows 0 and 1) in FP32 and 16 bits, where bandwidth bounds the dslash; FP64
// and double-float keep all 18 reals: their dslash is bound by arithmetic (GB300's FP64 pipe is a
// small fraction of its FP32 pipe, double-float costs ~10 FP32 operations per operation), and the
// row-2 reconstruction would cost about a fifth of their arithmetic to save bandwidth they do not use
inline size_t gauge_link_bytes(int prec) { return wide(prec) ? 144 : (prec == P_F32 ? 48 : 24); }
template <int P>
__host__ __device__ constexpr size_t gauge_link_bytes_dev()
{
    return (P == P_DF64 || P == P_F64) ? 144 : (P == P_F32 ? 48 : 24);
}
template <int P>
__host__ __device__ constexpr int nchunk_dev() { return (P == P_F64 || P == P_DF64) ? 12 : (P == P_F32 ? 6 : 3); }

// ---------------------------------------------------------------------------
// double-float arithmetic (Dekker / Knuth error-free transformations)
// ---------------------------------------------------------------------------
struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr df64(float f) : hi(f), lo(0.f) {}
    __host__ __device__ constexpr df64(int i) : hi((float)i), lo(0.f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ df64 df_renorm(float s, float e)
{
    const float hi = s + e;
    return df64(hi, e - (hi - s));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    const float s = a.hi + b.hi;
    const float v = s - a.hi;
    float e = (a.hi - (s - v)) + (b.hi - v);  // two-sum error
    e += a.lo + b.lo;
    return df_renorm(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);  // two-product error
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_renorm(p, e);
}
__device__ __forceinline__ df64 operator*(float a, df64 b)
{
    const float p = a * b.hi;
    float e = fmaf(a, b.hi, -p);
    e = fmaf(a, b.lo, e);
    return df_renorm(p, e);
}
__device__ __forceinline__ df64 operator*(int s, df64 b)
{
    if (s == 1) return b;
    if (s == -1) return -b;
    return (float)s * b;
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

// Nanoseconds of the GPU's global timer (bounds the wall time of every spin-wait).
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // 2 s

// Division of a non-negative 31-bit integer by a divisor fixed at set-up, by one
// high multiply, an add and a shift (Granlund and Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994, Thm. 4.2 with N = 32):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, q = (mulhi(m, n) + n) >> l.
// mulhi(m, n) < n, so the sum stays below 2^32 for n < 2^31.
struct FastDiv {
    uint32_t d, m, l;
    FastDiv() = default;
    explicit FastDiv(uint32_t div) : d(div), m(0), l(0)
    {
        while ((1ull << l) < div) ++l;
        m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1);
    }
    __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const
    {
#ifdef __CUDA_ARCH__
        const uint32_t hi = __umulhi(m, n);
#else
        const uint32_t hi = (uint32_t)(((uint64_t)m * n) >> 32);
#endif
        return (hi + n) >> l;
    }
};

struct Geom {
    int L[4];   // Lx, Ly, Lz, Lt
    int Lxh;    // Lx / 2
    int Vh;     // sites per parity
    double bc[4];
    float fbc[4];         // the same phases for FP32 arithmetic (no FP64 conversion in the kernels)
    FastDiv fxh, fy, fz;  // division by Lxh, Ly, Lz
};

// A host double in the kernel's arithmetic type: FP32 kernels read a copy made on the host,
// so that they issue no FP64 conversion (GB300's FP64 pipe is narrow).
template <typename Real>
__device__ __forceinline__ Real coef(double d, float f)
{
    if constexpr (std::is_same<Real, float>::value)
        return f;
    else
        return (Real)d;
}

// A field of nrhs right-hand sides in the internal layout of one precision.
struct FieldDesc {
    int prec;
    int nrhs;
    int Vh;
    char* data;   // [nrhs][2][NCH][Vh] x 16 bytes
    float* norm;  // [nrhs][2][Vh] (16-bit formats), else null
    size_t parity_bytes() const { return (size_t)spinor_chunks(prec) * 16 * Vh; }
    size_t rhs_bytes() const { return 2 * parity_bytes(); }
    char* ptr(int r, int p) const { return data + r * rhs_bytes() + p * parity_bytes(); }
    float* nptr(int r, int p) const { return norm ? norm + ((size_t)r * 2 + p) * Vh : nullptr; }
};

// ---------------------------------------------------------------------------
// geometry on the device
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cb_coords(const Geom& g, int s, int p, int c[4])
{
    const uint32_t r0 = g.fxh.div((uint32_t)s);
    const int xh = s - (int)r0 * g.Lxh;
    const uint32_t r1 = g.fy.div(r0);
    c[1] = (int)(r0 - r1 * (uint32_t)g.L[1]);
    const uint32_t r2 = g.fz.div(r1);
    c[2] = (int)(r1 - r2 * (uint32_t)g.L[2]);
    c[3] = (int)r2;
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}

__device__ __forceinline__ int cb_index(const Geom& g, int x, int y, int z, int t)
{
    return ((t * g.L[2] + z) * g.L[1] + y) * g.Lxh + (x >> 1);
}

// Checkerboard indices of the eight neighbours of site s (coordinates c), in the
// order +x, -x, +y, -y, +z, -z, +t, -t, as offsets from s: both parities number
// their sites the same way, so a y, z or t hop is a fixed shift (with the
// periodic wrap), and an x hop stays in the row of s.
template <int H>
__device__ __forceinline__ int cb_neighbour(const Geom& g, int s, const int c[4])
{
    const int dy = g.Lxh, dz = g.Lxh * g.L[1], dt = dz * g.L[2];
    if constexpr (H == 0) return s - (c[0] >> 1) + ((c[0] + 1 == g.L[0] ? 0 : c[0] + 1) >> 1);
    if constexpr (H == 1) return s - (c[0] >> 1) + ((c[0] == 0 ? g.L[0] - 1 : c[0] - 1) >> 1);
    if constexpr (H == 2) return c[1] + 1 == g.L[1] ? s - (g.L[1] - 1) * dy : s + dy;
    if constexpr (H == 3) return c[1] == 0 ? s + (g.L[1] - 1) * dy : s - dy;
    if constexpr (H == 4) return c[2] + 1 == g.L[2] ? s - (g.L[2] - 1) * dz : s + dz;
    if constexpr (H == 5) return c[2] == 0 ? s + (g.L[2] - 1) * dz : s - dz;
    if constexpr (H == 6) return c[3] + 1 == g.L[3] ? s - (g.L[3] - 1) * dt : s + dt;
    return c[3] == 0 ? s + (g.L[3] - 1) * dt : s - dt;
}

__device__ __forceinline__ void cb_neighbours(const Geom& g, int s, const int c[4], int nb[8])
{
    const int row = s - (c[0] >> 1);
    const int xp = c[0] + 1 == g.L[0] ? 0 : c[0] + 1;
    const int xm = c[0] == 0 ? g.L[0] - 1 : c[0] - 1;
    nb[0] = row + (xp >> 1);
    nb[1] = row + (xm >> 1);
    const int dy = g.Lxh, dz = g.Lxh * g.L[1], dt = dz * g.L[2];
    nb[2] = c[1] + 1 == g.L[1] ? s - (g.L[1] - 1) * dy : s + dy;
    nb[3] = c[1] == 0 ? s + (g.L[1] - 1) * dy : s - dy;
    nb[4] = c[2] + 1 == g.L[2] ? s - (g.L[2] - 1) * dz : s + dz;
    nb[5] = c[2] == 0 ? s + (g.L[2] - 1) * dz : s - dz;
    nb[6] = c[3] + 1 == g.L[3] ? s - (g.L[3] - 1) * dt : s + dt;
    nb[7] = c[3] == 0 ? s + (g.L[3] - 1) * dt : s - dt;
}

// ---------------------------------------------------------------------------
// 16-bit helpers
// ---------------------------------------------------------------------------
template <int P> struct Half;
template <> struct Half<P_F16> {
    __device__ static __forceinline__ float2 to2(uint32_t w)
    {
        __half2 h = *reinterpret_cast<__half2*>(&w);
        return __half22float2(h);
    }
    __device__ static __forceinline__ uint32_t from2(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
};
template <> struct Half<P_BF16> {
    __device__ static __forceinline__ float2 to2(uint32_t w)
    {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
        return __bfloat1622float2(h);
    }
    __device__ static __forceinline__ uint32_t from2(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
};

// ---------------------------------------------------------------------------
// spinor load / store: v[24] = (spin, colour, re/im)
// `base` points at chunk 0 of one (rhs, parity); `nrm` at its norm array.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R from_df(df64 a)
{
    if constexpr (std::is_same<R, df64>::value)
        return a;
    else
        return (R)a;
}
template <typename R>
__device__ __forceinline__ df64 to_df(R v)
{
    if constexpr (std::is_same<R, df64>::value)
        return v;
    else
        return df64(v);
}

template <int P, typename Real>
__device__ __forceinline__ void load_spinor(const char* __restrict__ base, const float* __restrict__ nrm,
                                            int Vh, int s, Real v[24])
{
    if constexpr (P == P_DF64) {
        const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float4 t = __ldg(b + (size_t)k * Vh + s);
            v[2 * k] = from_df<Real>(df64(t.x, t.y));
            v[2 * k + 1] = from_df<Real>(df64(t.z, t.w));
        }
    } else if constexpr (P == P_F64) {
        const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 t = __ldg(b + (size_t)k * Vh + s);
            v[2 * k] = (Real)t.x;
            v[2 * k + 1] = (Real)t.y;
        }
    } else if constexpr (P == P_F32) {
        const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 t = __ldg(b + (size_t)k * Vh + s);
            v[4 * k] = t.x;
            v[4 * k + 1] = t.y;
            v[4 * k + 2] = t.z;
            v[4 * k + 3] = t.w;
        }
    } else {
        const uint4* b = reinterpret_cast<const uint4*>(base);
        float n = __ldg(nrm + s);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 t = __ldg(b + (size_t)k * Vh + s);
            float2 a0 = Half<P>::to2(t.x), a1 = Half<P>::to2(t.y), a2 = Half<P>::to2(t.z),
                   a3 = Half<P>::to2(t.w);
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

// 16-bit storage: the 24 stored values without their site scale, which is returned
template <int P>
__device__ __forceinline__ float load_spinor_unscaled(const char* __restrict__ base, const float* __restrict__ nrm,
                                                      int Vh, int s, float v[24])
{
    const uint4* b = reinterpret_cast<const uint4*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint4 t = __ldg(b + (size_t)k * Vh + s);
        const float2 a0 = Half<P>::to2(t.x), a1 = Half<P>::to2(t.y), a2 = Half<P>::to2(t.z), a3 = Half<P>::to2(t.w);
        v[8 * k + 0] = a0.x;
        v[8 * k + 1] = a0.y;
        v[8 * k + 2] = a1.x;
        v[8 * k + 3] = a1.y;
        v[8 * k + 4] = a2.x;
        v[8 * k + 5] = a2.y;
        v[8 * k + 6] = a3.x;
        v[8 * k + 7] = a3.y;
    }
    return __ldg(nrm + s);
}

template <int P, typename Real>
__device__ __forceinline__ void store_spinor(char* __restrict__ base, float* __restrict__ nrm, int Vh, int s,
                                             const Real v[24])
{
    if constexpr (P == P_DF64) {
        float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const df64 a = to_df<Real>(v[2 * k]), c = to_df<Real>(v[2 * k + 1]);
            b[(size_t)k * Vh + s] = make_float4(a.hi, a.lo, c.hi, c.lo);
        }
    } else if constexpr (P == P_F64) {
        double2* b = reinterpret_cast<double2*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) b[(size_t)k * Vh + s] = make_double2((double)v[2 * k], (double)v[2 * k + 1]);
    } else if constexpr (P == P_F32) {
        float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            b[(size_t)k * Vh + s] =
                make_float4((float)v[4 * k], (float)v[4 * k + 1], (float)v[4 * k + 2], (float)v[4 * k + 3]);
    } else {
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < 24; ++i) m = fmaxf(m, fabsf((float)v[i]));
        float inv = m > 0.f ? 1.0f / m : 0.f;
        uint4* b = reinterpret_cast<uint4*>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 t;
            t.x = Half<P>::from2((float)v[8 * k + 0] * inv, (float)v[8 * k + 1] * inv);
            t.y = Half<P>::from2((float)v[8 * k + 2] * inv, (float)v[8 * k + 3] * inv);
            t.z = Half<P>::from2((float)v[8 * k + 4] * inv, (float)v[8 * k + 5] * inv);
            t.w = Half<P>::from2((float)v[8 * k + 6] * inv, (float)v[8 * k + 7] * inv);
            b[(size_t)k * Vh + s] = t;
        }
        nrm[s] = m;
    }
}

// ---------------------------------------------------------------------------
// gauge link load with reconstruct-12: u[18] = 3x3 complex, row-major
// `base` points at link[p][mu] chunk 0.
// ---------------------------------------------------------------------------
template <int P, typename Real>
__device__ __forceinline__ void load_link_rows(const char* __restrict__ base, int Vh, int s, Real u[18])
{
    if constexpr (P == P_DF64) {
        const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 t = __ldg(b + (size_t)k * Vh + s);
            u[2 * k] = from_df<Real>(df64(t.x, t.y));
            u[2 * k + 1] = from_df<Real>(df64(t.z, t.w));
        }
    } else if constexpr (P == P_F64) {
        const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double2 t = __ldg(b + (size_t)k * Vh + s);
            u[2 * k] = (Real)t.x;
            u[2 * k + 1] = (Real)t.y;
        }
    } else if constexpr (P == P_F32) {
        const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 t = __ldg(b + (size_t)k * Vh + s);
            u[4 * k] = t.x;
            u[4 * k + 1] = t.y;
            u[4 * k + 2] = t.z;
            u[4 * k + 3] = t.w;
        }
    } else {
        const uint2* b = reinterpret_cast<const uint2*>(base);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint2 t = __ldg(b + (size_t)k * Vh + s);
            float2 a0 = Half<P>::to2(t.x), a1 = Half<P>::to2(t.y);
            u[4 * k] = a0.x;
            u[4 * k + 1] = a0.y;
            u[4 * k + 2] = a1.x;
            u[4 * k + 3] = a1.y;
        }
    }
}

// row 2 = conj(row0 x row1)  (unitarity and det = 1)
template <typename Real>
__device__ __forceinline__ Real fma_any(Real a, Real b, Real c)
{
    if constexpr (std::is_same<Real, df64>::value)
        return a * b + c;
    else
        return fma(a, b, c);
}
template <typename Real>
__device__ __forceinline__ void link_row2(Real u[18])
{
    // (r0 x r1)_0 = r0_1 r1_2 - r0_2 r1_1, _1 = r0_2 r1_0 - r0_0 r1_2, _2 = r0_0 r1_1 - r0_1 r1_0; each real
    // part one chain of a multiply and three fused multiply-adds
#define OV_RE(i) u[2 * (i)]
#define OV_IM(i) u[2 * (i) + 1]
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        int a = (j + 1) % 3, b = (j + 2) % 3;
        // r0_a r1_b - r0_b r1_a
        Real re = OV_IM(b) * OV_IM(3 + a);
        re = fma_any<Real>(-OV_RE(b), OV_RE(3 + a), re);
        re = fma_any<Real>(-OV_IM(a), OV_IM(3 + b), re);
        re = fma_any<Real>(OV_RE(a), OV_RE(3 + b), re);
        Real im = -(OV_IM(b) * OV_RE(3 + a));
        im = fma_any<Real>(-OV_RE(b), OV_IM(3 + a), im);
        im = fma_any<Real>(OV_IM(a), OV_RE(3 + b), im);
        im = fma_any<Real>(OV_RE(a), OV_IM(3 + b), im);
        u[12 + 2 * j] = re;
        u[12 + 2 * j + 1] = -im;
    }
#undef OV_RE
#undef OV_IM
}

template <int P, typename Real>
__device__ __forceinline__ void load_link(const char* __restrict__ base, int Vh, int s, Real u[18])
{
    load_link_rows<P, Real>(base, Vh, s, u);
    if constexpr (P == P_DF64) {  // stored third row (9 chunks per link)
        const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int k = 6; k < 9; ++k) {
            float4 t = __ldg(b + (size_t)k * Vh + s);
            u[2 * k] = from_df<Real>(df64(t.x, t.y));
            u[2 * k + 1] = from_df<Real>(df64(t.z, t.w));
        }
    } else if constexpr (P == P_F64) {  // stored third row (9 chunks per link)
        const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
        for (int k = 6; k < 9; ++k) {
            double2 t = __ldg(b + (size_t)k * Vh + s);
            u[2 * k] = (Real)t.x;
            u[2 * k + 1] = (Real)t.y;
        }
    } else {
        link_row2<Real>(u);
    }
}

}  // namespace ov
