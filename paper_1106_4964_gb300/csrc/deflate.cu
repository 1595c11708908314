// Low-mode projection kernels (Eqs. 6-7 and 9 of the paper):
//   c[i][r]  = eta_i^dag psi_r                       (proj_dots + proj_finalize)
//   out1_r   = psi_r - sum_i eta_i c[i][r]           (the high-mode part psi_h)
//   out2_r   = gamma5 sum_i s_i c[i][r] eta_i        (gamma5 of the exact low-mode sign)
// on the CUDA cores.  The eigenvectors are nev single-rhs fields stored back
// to back in one internal-layout allocation.  Each thread owns one site of
// one right-hand side; the right-hand sides of a block share every
// eigenvector load through L1, and each pass over the sites handles IB
// eigenvectors with register accumulators.
#include <type_traits>

#include "ov_internal.cuh"
#include "ov_kernels.h"

namespace ov {

namespace {

constexpr int IB = 16;       // eigenvectors per pass of proj_dots
constexpr int PD_BX = 32;    // sites per warp row

template <int P>
using dreal_t = typename std::conditional<P == P_F64, double, typename std::conditional<P == P_DF64, df64, float>::type>::type;

// grid (nblk, ceil(nev/IB)); block (32, BY) with y = r + nrhs * grp, BY = nrhs * G
// partials layout [nblk * G][nev][nrhs] (double2)
template <int PV, int PS>
__global__ void __launch_bounds__(512) proj_dots_kernel(Geom g, FieldDesc eta, int nev, FieldDesc psi, int G,
                                                        double2* partials)
{
    using Real = dreal_t<PS>;
    constexpr size_t CV = nchunk_dev<PV>() * 16, CS = nchunk_dev<PS>() * 16;
    const int R = psi.nrhs;
    const int r = threadIdx.y % R, grp = threadIdx.y / R;
    const int i0 = blockIdx.y * IB;
    const int N = 2 * g.Vh;
    const size_t eta_rhs = 2 * CV * g.Vh;
    Real accr[IB], acci[IB];
#pragma unroll
    for (int j = 0; j < IB; ++j) accr[j] = acci[j] = 0;
    const int stride = gridDim.x * G * PD_BX;
    for (int idx = (blockIdx.x * G + grp) * PD_BX + threadIdx.x; idx < N; idx += stride) {
        const int p = idx >= g.Vh, s = idx - p * g.Vh;
        Real a[24];
        const size_t rp = (size_t)r * 2 + p;
        load_spinor<PS, Real>(psi.data + rp * CS * g.Vh, psi.norm ? psi.norm + rp * g.Vh : nullptr, g.Vh, s, a);
#pragma unroll
        for (int j = 0; j < IB; ++j) {
            const int i = i0 + j;
            if (i < nev) {
                Real e[24];
                load_spinor<PV, Real>(eta.data + i * eta_rhs + p * CV * g.Vh,
                                      eta.norm ? eta.norm + ((size_t)i * 2 + p) * g.Vh : nullptr, g.Vh, s, e);
                Real tr = 0, ti = 0;
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    tr += e[2 * k] * a[2 * k] + e[2 * k + 1] * a[2 * k + 1];
                    ti += e[2 * k] * a[2 * k + 1] - e[2 * k + 1] * a[2 * k];
                }
                accr[j] += tr;
                acci[j] += ti;
            }
        }
    }
    const size_t part = (size_t)blockIdx.x * G + grp;
#pragma unroll
    for (int j = 0; j < IB; ++j) {
        double vr = (double)accr[j], vi = (double)acci[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, o);
            vi += __shfl_xor_sync(0xffffffffu, vi, o);
        }
        const int i = i0 + j;
        if (threadIdx.x == 0 && i < nev) partials[(part * nev + i) * R + r] = make_double2(vr, vi);
    }
}

__global__ void proj_finalize_kernel(const double2* partials, int nparts, int n, double2* out)
{
    // one thread per output element, fixed summation order
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double re = 0, im = 0;
    for (int b = 0; b < nparts; ++b) {
        double2 v = partials[(size_t)b * n + k];
        re += v.x;
        im += v.y;
    }
    out[k] = make_double2(re, im);
}

// grid (ceil(2Vh / BX)); block (BX, R)
template <int PV, int PS>
__global__ void __launch_bounds__(512) proj_update_kernel(Geom g, FieldDesc eta, int nev, const double2* c,
                                                          const double* sg, FieldDesc psi, FieldDesc out1,
                                                          FieldDesc out2)
{
    using Real = dreal_t<PS>;
    // coefficients in the arithmetic type (converted once per block, not once per site):
    // (re, im) pairs [nev][R] for out1, then [nev][R] for out2
    extern __shared__ __align__(16) unsigned char sh_raw[];
    Real* sh_c = reinterpret_cast<Real*>(sh_raw);
    const int R = psi.nrhs;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = tid; k < nev * R; k += blockDim.x * blockDim.y) {
        const double2 v = c[k];
        const double s = sg ? sg[k / R] : 0.0;
        sh_c[2 * k] = (Real)v.x;
        sh_c[2 * k + 1] = (Real)v.y;
        sh_c[2 * (nev * R + k)] = (Real)(s * v.x);
        sh_c[2 * (nev * R + k) + 1] = (Real)(s * v.y);
    }
    __syncthreads();
    constexpr size_t CV = nchunk_dev<PV>() * 16, CS = nchunk_dev<PS>() * 16;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = threadIdx.y;
    if (idx >= 2 * g.Vh || r >= R) return;
    const int p = idx >= g.Vh, s = idx - p * g.Vh;
    const size_t eta_rhs = 2 * CV * g.Vh;
    Real o1[24], o2[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) o1[k] = o2[k] = 0;
    const bool want2 = out2.data != nullptr;
    for (int i = 0; i < nev; ++i) {
        Real e[24];
        load_spinor<PV, Real>(eta.data + i * eta_rhs + p * CV * g.Vh,
                              eta.norm ? eta.norm + ((size_t)i * 2 + p) * g.Vh : nullptr, g.Vh, s, e);
        const Real cr = sh_c[2 * (i * R + r)], ci = sh_c[2 * (i * R + r) + 1];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            o1[2 * k] += cr * e[2 * k] - ci * e[2 * k + 1];
            o1[2 * k + 1] += cr * e[2 * k + 1] + ci * e[2 * k];
        }
        if (want2) {
            const Real dr = sh_c[2 * (nev * R + i * R + r)], di = sh_c[2 * (nev * R + i * R + r) + 1];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                o2[2 * k] += dr * e[2 * k] - di * e[2 * k + 1];
                o2[2 * k + 1] += dr * e[2 * k + 1] + di * e[2 * k];
            }
        }
    }
    const size_t rp = (size_t)r * 2 + p;
    Real a[24];
    load_spinor<PS, Real>(psi.data + rp * CS * g.Vh, psi.norm ? psi.norm + rp * g.Vh : nullptr, g.Vh, s, a);
#pragma unroll
    for (int k = 0; k < 24; ++k) a[k] -= o1[k];
    store_spinor<PS, Real>(out1.data + rp * CS * g.Vh, out1.norm ? out1.norm + rp * g.Vh : nullptr, g.Vh, s, a);
    if (want2) {
#pragma unroll
        for (int k = 12; k < 24; ++k) o2[k] = -o2[k];
        store_spinor<PS, Real>(out2.data + rp * CS * g.Vh, out2.norm ? out2.norm + rp * g.Vh : nullptr, g.Vh, s,
                               o2);
    }
}

int groups_for(int R) { return R >= 8 ? 1 : (R >= 4 ? 2 : (R >= 2 ? 4 : 8)); }

template <int PV, int PS>
cudaError_t dots2(const Geom& g, const FieldDesc& eta, int nev, const FieldDesc& psi, double2* partials, int nblk,
                  cudaStream_t st)
{
    const int G = groups_for(psi.nrhs);
    dim3 block(PD_BX, psi.nrhs * G);
    dim3 grid(nblk, (nev + IB - 1) / IB);
    proj_dots_kernel<PV, PS><<<grid, block, 0, st>>>(g, eta, nev, psi, G, partials);
    return cudaGetLastError();
}

template <int PV, int PS>
cudaError_t update2(const Geom& g, const FieldDesc& eta, int nev, const double2* c, const double* s,
                    const FieldDesc& psi, const FieldDesc& out1, const FieldDesc& out2, cudaStream_t st)
{
    const int R = psi.nrhs;
    const int bx = R >= 8 ? 32 : (R >= 4 ? 64 : 128);
    dim3 block(bx, R);
    dim3 grid((2 * g.Vh + bx - 1) / bx);
    size_t shm = 4 * sizeof(dreal_t<PS>) * nev * R;
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(proj_update_kernel<PV, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)shm);
        if (e != cudaSuccess) return e;
    }
    proj_update_kernel<PV, PS><<<grid, block, shm, st>>>(g, eta, nev, c, s, psi, out1, out2);
    return cudaGetLastError();
}

}  // namespace

int proj_groups(int nrhs) { return groups_for(nrhs); }

cudaError_t launch_proj_dots(const Geom& g, const FieldDesc& eta, int nev, const FieldDesc& psi, double2* partials,
                             int nblk, cudaStream_t st)
{
    if (psi.nrhs * groups_for(psi.nrhs) * PD_BX > 512) return cudaErrorInvalidValue;
    int pv = eta.prec, ps = psi.prec;
    if (pv == P_F64 && ps == P_F64) return dots2<P_F64, P_F64>(g, eta, nev, psi, partials, nblk, st);
    if (pv == P_DF64 && ps == P_DF64) return dots2<P_DF64, P_DF64>(g, eta, nev, psi, partials, nblk, st);
    if (pv == P_F32 && ps == P_F32) return dots2<P_F32, P_F32>(g, eta, nev, psi, partials, nblk, st);
    if (pv == P_F16 && ps == P_F32) return dots2<P_F16, P_F32>(g, eta, nev, psi, partials, nblk, st);
    if (pv == P_BF16 && ps == P_F32) return dots2<P_BF16, P_F32>(g, eta, nev, psi, partials, nblk, st);
    if (pv == P_F16 && ps == P_F16) return dots2<P_F16, P_F16>(g, eta, nev, psi, partials, nblk, st);
    if (pv == P_BF16 && ps == P_BF16) return dots2<P_BF16, P_BF16>(g, eta, nev, psi, partials, nblk, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_proj_finalize(const double2* partials, int nparts, int n, double2* out, cudaStream_t st)
{
    proj_finalize_kernel<<<(n + 127) / 128, 128, 0, st>>>(partials, nparts, n, out);
    return cudaGetLastError();
}

cudaError_t launch_proj_update(const Geom& g, const FieldDesc& eta, int nev, const double2* c, const double* s,
                               const FieldDesc& psi, const FieldDesc& out1, const FieldDesc& out2, cudaStream_t st)
{
    if (psi.nrhs > 16) return cudaErrorInvalidValue;
    int pv = eta.prec, ps = psi.prec;
    if (pv == P_F64 && ps == P_F64) return update2<P_F64, P_F64>(g, eta, nev, c, s, psi, out1, out2, st);
    if (pv == P_DF64 && ps == P_DF64) return update2<P_DF64, P_DF64>(g, eta, nev, c, s, psi, out1, out2, st);
    if (pv == P_F32 && ps == P_F32) return update2<P_F32, P_F32>(g, eta, nev, c, s, psi, out1, out2, st);
    if (pv == P_F16 && ps == P_F32) return update2<P_F16, P_F32>(g, eta, nev, c, s, psi, out1, out2, st);
    if (pv == P_BF16 && ps == P_F32) return update2<P_BF16, P_F32>(g, eta, nev, c, s, psi, out1, out2, st);
    if (pv == P_F16 && ps == P_F16) return update2<P_F16, P_F16>(g, eta, nev, c, s, psi, out1, out2, st);
    if (pv == P_BF16 && ps == P_BF16) return update2<P_BF16, P_BF16>(g, eta, nev, c, s, psi, out1, out2, st);
    return cudaErrorInvalidValue;
}

}  // namespace ov
