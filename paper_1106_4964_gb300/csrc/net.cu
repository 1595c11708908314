// Learned gauge-covariant preconditioner (no counterpart in the paper).
//
// Layer (channels cin -> cout):
//   y_c(n) = sum_{c'} sum_{p=0..8} W[p][c][c'] (T_p x_{c'})(n)
// with T_0 = 1, T_{1+2mu} x(n) = U_mu(n) x(n+mu), T_{2+2mu} x(n) = U_mu(n-mu)^dag x(n-mu)
// (boundary phases applied) and W[p][c][c'] a complex 4x4 spin matrix.  The
// map is linear and commutes with gauge transformations.  The network is
// M = L2 . L1 with 1 -> 16 -> 1 channels, applied to one right-hand side
// at a time in FP32 (internal even/odd layout; activations are 16-rhs fields).
//
// Backward pass: the adjoint of T_p is T_{pbar} (forward <-> backward hop),
// so the input gradient is the forward kernel with weights
// W'[q][c'][c] = W[qbar][c][c']^dag; the weight gradient
// gW[p][c][c'] = sum_n gy_c(n) (T_p x_{c'}(n))^dag (summed over colour) is a
// split-K reduction over sites with block partials summed in fixed order.
// Training: loss sum_k |M(r_k) - e_k|^2 / |e_k|^2 over (residual, error)
// pairs recorded at the FP64 true-residual points of the library's own
// deflated CG solves, Adam on the device.
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"

namespace ov {

constexpr int NET_C = 16;              // hidden channels
constexpr int NET_W = 9 * NET_C * 16;  // complex weights per layer (9 paths x 16 ch x 4x4 spin)
constexpr int NET_PARAMS = 2 * NET_W;  // complex parameters of the network
constexpr int NET_MAXPAIRS = 256;

struct NetState {
    int trained = 0;
    float2* W = nullptr;     // layer 1 [9][16][1][16] then layer 2 [9][1][16][16]
    float2* Wadj = nullptr;  // adjoint weights, same layout per layer with channels swapped
    float2* G = nullptr;     // gradient
    float* adam = nullptr;   // first moments [2*NET_PARAMS] then second moments
    float2* partials = nullptr;
    size_t partials_n = 0;
    int adam_t = 0;
    int adj_valid = 0;  // Wadj matches W
    // recorded training pairs: residuals and iterates (then errors), f32 single-rhs fields
    int recording = 0;
    FieldDesc pr{}, px{};
    int npairs = 0, cap = 0;
    std::vector<double> history;  // mean loss per pair before each Adam step of the last training
};

namespace {

struct PathSite {
    int sn, q;        // source checkerboard site and parity
    float u[18];      // link (forward: U, backward: U used as U^dag)
    float ph;
};

__device__ __forceinline__ void path_setup(const Geom& g, const char* gauge, int p, int s, const int c[4], int path,
                                           PathSite& P)
{
    if (path == 0) {
        P.sn = s;
        P.q = p;
        P.ph = 1.f;
        return;
    }
    const int mu = (path - 1) >> 1;
    const bool fwd = ((path - 1) & 1) == 0;
    int d[4] = {c[0], c[1], c[2], c[3]};
    bool cross;
    if (fwd) {
        d[mu] = c[mu] + 1 == g.L[mu] ? 0 : c[mu] + 1;
        cross = d[mu] == 0;
    } else {
        d[mu] = c[mu] == 0 ? g.L[mu] - 1 : c[mu] - 1;
        cross = c[mu] == 0;
    }
    P.sn = cb_index(g, d[0], d[1], d[2], d[3]);
    P.q = 1 - p;
    const int lpar = fwd ? p : P.q, ls = fwd ? s : P.sn;
    load_link<P_F32, float>(gauge + ((size_t)(lpar * 4 + mu) * g.Vh) * 48, g.Vh, ls, P.u);
    P.ph = cross ? (float)g.bc[mu] : 1.f;
}

// t = T_path x_c (one channel; xc = channel base, both parities)
__device__ __forceinline__ void path_apply(const Geom& g, const char* xc, int path, const PathSite& P, float t[24])
{
    const size_t par = (size_t)6 * 16 * g.Vh;
    float v[24];
    load_spinor<P_F32, float>(xc + P.q * par, nullptr, g.Vh, P.sn, v);
    if (path == 0) {
#pragma unroll
        for (int k = 0; k < 24; ++k) t[k] = v[k];
        return;
    }
    const bool fwd = ((path - 1) & 1) == 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float re = 0, im = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float ur = fwd ? P.u[2 * (3 * i + j)] : P.u[2 * (3 * j + i)];
                float ui = fwd ? P.u[2 * (3 * i + j) + 1] : -P.u[2 * (3 * j + i) + 1];
                float xr = v[2 * (3 * s + j)], xi = v[2 * (3 * s + j) + 1];
                re += ur * xr - ui * xi;
                im += ur * xi + ui * xr;
            }
            t[2 * (3 * s + i)] = P.ph * re;
            t[2 * (3 * s + i) + 1] = P.ph * im;
        }
}

// forward layer: thread per (site, group of CG output channels); W in shared memory
template <int CIN, int COUT, int CG>
__global__ void __launch_bounds__(128) net_fwd_kernel(Geom g, const char* gauge, const char* x, char* y,
                                                      const float2* __restrict__ Wg)
{
    __shared__ float2 W[9 * COUT * CIN * 16];
    for (int k = threadIdx.x; k < 9 * COUT * CIN * 16; k += blockDim.x) W[k] = Wg[k];
    __syncthreads();
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int grp = blockIdx.y;
    if (idx >= 2 * g.Vh) return;
    const int p = idx >= g.Vh, s = idx - p * g.Vh;
    int c[4];
    cb_coords(g, s, p, c);
    const size_t chan = (size_t)2 * 6 * 16 * g.Vh;  // bytes of one single-rhs f32 field
    float acc[CG][24];
#pragma unroll
    for (int j = 0; j < CG; ++j)
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[j][k] = 0.f;
    for (int path = 0; path < 9; ++path) {
        PathSite P;
        path_setup(g, gauge, p, s, c, path, P);
        for (int ci = 0; ci < CIN; ++ci) {
            float t[24];
            path_apply(g, x + ci * chan, path, P, t);
#pragma unroll
            for (int j = 0; j < CG; ++j) {
                const float2* w = W + ((path * COUT + grp * CG + j) * CIN + ci) * 16;
#pragma unroll
                for (int sa = 0; sa < 4; ++sa)
#pragma unroll
                    for (int sb = 0; sb < 4; ++sb) {
                        const float2 ww = w[4 * sa + sb];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            float tr = t[2 * (3 * sb + a)], ti = t[2 * (3 * sb + a) + 1];
                            acc[j][2 * (3 * sa + a)] += ww.x * tr - ww.y * ti;
                            acc[j][2 * (3 * sa + a) + 1] += ww.x * ti + ww.y * tr;
                        }
                    }
            }
        }
    }
    const size_t par = (size_t)6 * 16 * g.Vh;
#pragma unroll
    for (int j = 0; j < CG; ++j)
        store_spinor<P_F32, float>(y + (grp * CG + j) * chan + p * par, nullptr, g.Vh, s, acc[j]);
}

// weight-gradient partials for path blockIdx.y over the block's sites,
// entry e = ((co * CIN + ci) * 16) + 4 * sa + sb
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) net_wgrad_kernel(Geom g, const char* gauge, const char* x, const char* gy,
                                                        float2* partials)
{
    constexpr int NS = 16;  // sites per staged chunk
    __shared__ float sg[COUT][NS][24];
    __shared__ float st[CIN][NS][24];
    const int path = blockIdx.y;
    const int e = threadIdx.x;
    const int co = e / (CIN * 16), ci = (e / 16) % CIN, sa = (e % 16) / 4, sb = e % 4;
    const bool active = e < COUT * CIN * 16;
    const size_t chan = (size_t)2 * 6 * 16 * g.Vh;
    const size_t par = (size_t)6 * 16 * g.Vh;
    double dr = 0, di = 0;
    const int N = 2 * g.Vh;
    for (int base = blockIdx.x * NS; base < N; base += gridDim.x * NS) {
        __syncthreads();
        for (int k = threadIdx.x; k < NS * (COUT + CIN); k += blockDim.x) {
            const int j = k % NS, ch = k / NS;
            const int idx = base + j;
            float v[24];
            if (idx < N) {
                const int p = idx >= g.Vh, s = idx - p * g.Vh;
                if (ch < COUT) {
                    load_spinor<P_F32, float>(gy + ch * chan + p * par, nullptr, g.Vh, s, v);
                } else {
                    int c[4];
                    cb_coords(g, s, p, c);
                    PathSite P;
                    path_setup(g, gauge, p, s, c, path, P);
                    path_apply(g, x + (ch - COUT) * chan, path, P, v);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 24; ++q) v[q] = 0.f;
            }
            float* dst = ch < COUT ? sg[ch][j] : st[ch - COUT][j];
#pragma unroll
            for (int q = 0; q < 24; ++q) dst[q] = v[q];
        }
        __syncthreads();
        if (active) {
            float accr = 0.f, acci = 0.f;
            for (int j = 0; j < NS; ++j)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float gr = sg[co][j][2 * (3 * sa + a)], gi = sg[co][j][2 * (3 * sa + a) + 1];
                    float tr = st[ci][j][2 * (3 * sb + a)], ti = st[ci][j][2 * (3 * sb + a) + 1];
                    accr += gr * tr + gi * ti;  // gy * conj(t)
                    acci += gi * tr - gr * ti;
                }
            dr += accr;
            di += acci;
        }
    }
    if (active)
        partials[((size_t)path * gridDim.x + blockIdx.x) * (COUT * CIN * 16) + e] = make_float2((float)dr, (float)di);
}

// gW[path][ent] (+)= sum_b partials[path][b][ent], fixed order
__global__ void net_wgrad_reduce(const float2* partials, int nblk, int nent, float2* gW, int accumulate)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 9 * nent) return;
    const int path = k / nent, ent = k % nent;
    double r = 0, i = 0;
    for (int b = 0; b < nblk; ++b) {
        float2 v = partials[((size_t)path * nblk + b) * nent + ent];
        r += v.x;
        i += v.y;
    }
    float2 o = make_float2((float)r, (float)i);
    if (accumulate) {
        o.x += gW[k].x;
        o.y += gW[k].y;
    }
    gW[k] = o;
}

// W'[q][c'][c] = W[qbar][c][c']^dag for a layer W[9][cout][cin][16]
__global__ void net_adjoint_weights(const float2* W, float2* Wa, int cin, int cout)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 9 * cout * cin * 16) return;
    const int q = k / (cin * cout * 16);
    int rem = k % (cin * cout * 16);
    const int cp = rem / (cout * 16);  // adjoint output channel = W input channel
    rem %= cout * 16;
    const int cc = rem / 16;           // adjoint input channel = W output channel
    const int e = rem % 16, sa = e / 4, sb = e % 4;
    const int qbar = q == 0 ? 0 : (((q - 1) & 1) ? q - 1 : q + 1);
    const float2 w = W[((qbar * cout + cc) * cin + cp) * 16 + 4 * sb + sa];
    Wa[k] = make_float2(w.x, -w.y);
}

__global__ void adam_kernel(float2* W, const float2* G, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2, float gscale)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * n) return;
    float* w = reinterpret_cast<float*>(W);
    const float gk = reinterpret_cast<const float*>(G)[k] * gscale;
    m[k] = b1 * m[k] + (1 - b1) * gk;
    v[k] = b2 * v[k] + (1 - b2) * gk * gk;
    w[k] -= lr * (m[k] / c1) / (sqrtf(v[k] / c2) + eps);
}

FieldDesc one(const FieldDesc& f, int i)
{
    FieldDesc s = f;
    s.nrhs = 1;
    s.data = f.data + (size_t)i * f.rhs_bytes();
    s.norm = f.norm ? f.norm + (size_t)i * 2 * f.Vh : nullptr;
    return s;
}

int net_init(ov_ctx* c)
{
    if (c->net) return OV_OK;
    NetState* n = new NetState();
    c->net = n;
    void* p = nullptr;
    OV_TRY(dev_alloc(c, &p, sizeof(float2) * NET_PARAMS));
    n->W = (float2*)p;
    OV_TRY(dev_alloc(c, &p, sizeof(float2) * NET_PARAMS));
    n->Wadj = (float2*)p;
    OV_TRY(dev_alloc(c, &p, sizeof(float2) * NET_PARAMS));
    n->G = (float2*)p;
    OV_TRY(dev_alloc(c, &p, sizeof(float) * 4 * NET_PARAMS));
    n->adam = (float*)p;
    OV_CUDA(c, cudaMemset(n->adam, 0, sizeof(float) * 4 * NET_PARAMS));
    OV_CUDA(c, cudaMemset(n->W, 0, sizeof(float2) * NET_PARAMS));
    return OV_OK;
}

int layer_fwd(ov_ctx* c, int layer, bool adj, const FieldDesc& x, const FieldDesc& y, cudaStream_t st)
{
    NetState* n = c->net;
    const float2* W = (adj ? n->Wadj : n->W) + (size_t)layer * NET_W;
    const Geom& g = c->g;
    const char* gauge = (const char*)c->gauge[P_F32];
    // layer 0: 1 -> 16 (adjoint 16 -> 1); layer 1: 16 -> 1 (adjoint 1 -> 16)
    const bool one_to_many = (layer == 0) != adj;
    if (one_to_many) {
        dim3 grid((2 * g.Vh + 127) / 128, NET_C / 4);
        net_fwd_kernel<1, NET_C, 4><<<grid, 128, 0, st>>>(g, gauge, x.data, y.data, W);
    } else {
        dim3 grid((2 * g.Vh + 127) / 128, 1);
        net_fwd_kernel<NET_C, 1, 1><<<grid, 128, 0, st>>>(g, gauge, x.data, y.data, W);
    }
    OV_CUDA(c, cudaGetLastError());
    return OV_OK;
}

int refresh_adjoint(ov_ctx* c, cudaStream_t st)
{
    NetState* n = c->net;
    net_adjoint_weights<<<(NET_W + 255) / 256, 256, 0, st>>>(n->W, n->Wadj, 1, NET_C);
    net_adjoint_weights<<<(NET_W + 255) / 256, 256, 0, st>>>(n->W + NET_W, n->Wadj + NET_W, NET_C, 1);
    OV_CUDA(c, cudaGetLastError());
    return OV_OK;
}

// loss over pairs k0..k1 of (pr, pe) and its gradient into n->G
int loss_grad(ov_ctx* c, const FieldDesc& pr, const FieldDesc& pe, int k0, int k1, double* loss, cudaStream_t st)
{
    NetState* n = c->net;
    const Geom& g = c->g;
    FieldDesc h, y, gy, gh;
    OV_TRY(ws_field(c, WS_NET_H, P_F32, NET_C, &h));
    OV_TRY(ws_field(c, WS_NET_GH, P_F32, NET_C, &gh));
    OV_TRY(ws_field(c, WS_NET_G, P_F32, 1, &y));
    OV_TRY(ws_field(c, WS_LZ_T, P_F32, 1, &gy));
    const int nblk = 2 * 152;
    const size_t need = (size_t)9 * nblk * 256;
    if (n->partials_n < need) {
        if (n->partials) {
            cudaDeviceSynchronize();
            dev_free(c, n->partials, sizeof(float2) * n->partials_n);
        }
        void* p = nullptr;
        OV_TRY(dev_alloc(c, &p, sizeof(float2) * need));
        n->partials = (float2*)p;
        n->partials_n = need;
    }
    OV_CUDA(c, cudaMemsetAsync(n->G, 0, sizeof(float2) * NET_PARAMS, st));
    OV_TRY(refresh_adjoint(c, st));
    const int np = k1 - k0;
    std::vector<double> en(np);
    double* dn = c->dscal + DSCAL_DOT;  // double2 per pair
    for (int k = k0; k < k1; ++k) OV_TRY(norm2(c, one(pe, k), dn + 2 * (k - k0), st));
    {
        std::vector<double2> h2(np);
        OV_CUDA(c, cudaMemcpyAsync(h2.data(), dn, sizeof(double2) * np, cudaMemcpyDeviceToHost, st));
        OV_CUDA(c, cudaStreamSynchronize(st));
        for (int k = 0; k < np; ++k) en[k] = h2[k].x > 0 ? h2[k].x : 1.0;
    }
    double* dg = c->dscal + DSCAL_NORM;
    for (int k = k0; k < k1; ++k) {
        FieldDesc r = one(pr, k), e = one(pe, k);
        OV_TRY(layer_fwd(c, 0, false, r, h, st));
        OV_TRY(layer_fwd(c, 1, false, h, y, st));
        // gy = 2 (y - e) / |e|^2, with |gy|^2 recorded for the loss
        FieldDesc xs[2] = {y, e};
        const double s2 = 2.0 / en[k - k0];
        double2 hc[2] = {make_double2(s2, 0), make_double2(-s2, 0)};
        OV_TRY(lincomb(c, gy, 2, xs, hc, nullptr, 0, dg + (k - k0), st));
        net_wgrad_kernel<NET_C, 1><<<dim3(nblk, 9), 256, 0, st>>>(g, (const char*)c->gauge[P_F32], h.data, gy.data,
                                                                  n->partials);
        net_wgrad_reduce<<<(9 * 256 + 255) / 256, 256, 0, st>>>(n->partials, nblk, 256, n->G + NET_W, 1);
        OV_TRY(layer_fwd(c, 1, true, gy, gh, st));  // gh = L2^dag gy
        net_wgrad_kernel<1, NET_C><<<dim3(nblk, 9), 256, 0, st>>>(g, (const char*)c->gauge[P_F32], r.data, gh.data,
                                                                  n->partials);
        net_wgrad_reduce<<<(9 * 256 + 255) / 256, 256, 0, st>>>(n->partials, nblk, 256, n->G, 1);
        OV_CUDA(c, cudaGetLastError());
    }
    std::vector<double> gn(np);
    OV_CUDA(c, cudaMemcpyAsync(gn.data(), dg, sizeof(double) * np, cudaMemcpyDeviceToHost, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    double total = 0;
    for (int k = 0; k < np; ++k) total += gn[k] * en[k] / 4.0;  // |y-e|^2/|e|^2 = |gy|^2 |e|^2 / 4
    *loss = total;
    return OV_OK;
}

}  // namespace

bool net_ready(const ov_ctx* c) { return c->net && c->net->trained; }

void net_free(ov_ctx* c)
{
    NetState* n = c->net;
    if (!n) return;
    cudaDeviceSynchronize();
    if (n->W) dev_free(c, n->W, sizeof(float2) * NET_PARAMS);
    if (n->Wadj) dev_free(c, n->Wadj, sizeof(float2) * NET_PARAMS);
    if (n->G) dev_free(c, n->G, sizeof(float2) * NET_PARAMS);
    if (n->adam) dev_free(c, n->adam, sizeof(float) * 4 * NET_PARAMS);
    if (n->partials) dev_free(c, n->partials, sizeof(float2) * n->partials_n);
    field_free(c, &n->pr);
    field_free(c, &n->px);
    delete n;
    c->net = nullptr;
}

// z = M r for every rhs of r (any precision; computed in FP32)
int net_apply_precond(ov_ctx* c, const FieldDesc& r, const FieldDesc& z, cudaStream_t st)
{
    if (!c->net) return set_err(c, OV_ESTATE, "learned preconditioner has no weights");
    NetState* n = c->net;
    const bool sym = c->net_sym != 0;
    if (sym && !n->adj_valid) {
        OV_TRY(refresh_adjoint(c, st));
        n->adj_valid = 1;
    }
    FieldDesc h, a, b, d;
    OV_TRY(ws_field(c, WS_NET_H, P_F32, NET_C, &h));
    OV_TRY(ws_field(c, WS_NET_G, P_F32, 1, &a));
    OV_TRY(ws_field(c, WS_NET_GH, P_F32, 1, &b));
    if (sym) OV_TRY(ws_field(c, WS_NET_S, P_F32, 1, &d));
    for (int q = 0; q < r.nrhs; ++q) {
        FieldDesc rq = one(r, q), zq = one(z, q);
        const bool f32in = r.prec == P_F32, f32out = z.prec == P_F32;
        if (!f32in) OV_TRY(convert(c, rq, a, st));
        const FieldDesc& x = f32in ? rq : a;
        OV_TRY(layer_fwd(c, 0, false, x, h, st));
        OV_TRY(layer_fwd(c, 1, false, h, (f32out && !sym) ? zq : b, st));
        if (sym) {
            // z = (M + M^dag) r / 2, M^dag = L1^dag L2^dag: Hermitian, as CG expects of a preconditioner
            OV_TRY(layer_fwd(c, 1, true, x, h, st));
            OV_TRY(layer_fwd(c, 0, true, h, d, st));
            FieldDesc v[2] = {b, d};
            double2 hc[2] = {make_double2(0.5, 0), make_double2(0.5, 0)};
            OV_TRY(lincomb(c, f32out ? zq : b, 2, v, hc, nullptr, 0, nullptr, st));
        }
        if (!f32out) OV_TRY(convert(c, b, zq, st));
    }
    return OV_OK;
}

// called by the CG at each FP64 true-residual point while recording
int net_record_pair(ov_ctx* c, const FieldDesc& r64, const FieldDesc& x64, cudaStream_t st)
{
    NetState* n = c->net;
    if (!n || !n->recording) return OV_OK;
    for (int q = 0; q < r64.nrhs && n->npairs < n->cap; ++q, ++n->npairs) {
        OV_TRY(convert(c, one(r64, q), one(n->pr, n->npairs), st));
        OV_TRY(convert(c, one(x64, q), one(n->px, n->npairs), st));
    }
    return OV_OK;
}

}  // namespace ov

using namespace ov;

extern "C" {

int ov_net_set_weights(ov_ctx* c, const double* w, int n)
{
    if (!c) return OV_EINVAL;
    if (!w || n != 2 * NET_PARAMS) return set_err(c, OV_EINVAL, "weights: expected %d doubles", 2 * NET_PARAMS);
    OV_TRY(net_init(c));
    std::vector<float2> h(NET_PARAMS);
    for (int i = 0; i < NET_PARAMS; ++i) h[i] = make_float2((float)w[2 * i], (float)w[2 * i + 1]);
    OV_CUDA(c, cudaMemcpy(c->net->W, h.data(), sizeof(float2) * NET_PARAMS, cudaMemcpyHostToDevice));
    c->net->trained = 1;
    c->net->adj_valid = 0;
    return OV_OK;
}

int ov_net_get_weights(ov_ctx* c, double* w, int n)
{
    if (!c) return OV_EINVAL;
    if (!w || n != 2 * NET_PARAMS) return set_err(c, OV_EINVAL, "weights: expected %d doubles", 2 * NET_PARAMS);
    if (!c->net) return set_err(c, OV_ESTATE, "no network weights");
    std::vector<float2> h(NET_PARAMS);
    OV_CUDA(c, cudaMemcpy(h.data(), c->net->W, sizeof(float2) * NET_PARAMS, cudaMemcpyDeviceToHost));
    for (int i = 0; i < NET_PARAMS; ++i) {
        w[2 * i] = h[i].x;
        w[2 * i + 1] = h[i].y;
    }
    return OV_OK;
}

int ov_net_apply(ov_ctx* c, const void* in, void* out, int nrhs, void* stream)
{
    if (!c) return OV_EINVAL;
    if (!in || !out || in == out) return set_err(c, OV_EINVAL, "bad buffers");
    if (nrhs < 1 || nrhs > 16) return set_err(c, OV_EINVAL, "nrhs out of range");
    if (!c->have_gauge) return set_err(c, OV_ESTATE, "no gauge field");
    if (!c->net) return set_err(c, OV_ESTATE, "no network weights");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)nrhs * 2 * c->g.Vh * 12 * 16;
    const double* din = nullptr;
    double* dout = nullptr;
    OV_TRY(stage_in(c, 0, in, bytes, st, &din));
    OV_TRY(stage_out_buffer(c, 1, out, bytes, &dout));
    FieldDesc fi, fo;
    OV_TRY(ws_field(c, WS_IN, P_F32, nrhs, &fi));
    OV_TRY(ws_field(c, WS_OUT, P_F32, nrhs, &fo));
    OV_CUDA(c, launch_pack(c->g, din, fi, 0, st));
    OV_TRY(net_apply_precond(c, fi, fo, st));
    OV_CUDA(c, launch_unpack(c->g, fo, dout, 0, st));
    return stage_out_finish(c, out, dout, bytes, st);
}

int ov_net_loss_grad(ov_ctx* c, const void* r, const void* e, int npairs, double* loss, double* grad, void* stream)
{
    if (!c) return OV_EINVAL;
    if (!r || !e || !loss || npairs < 1 || npairs > 16) return set_err(c, OV_EINVAL, "bad arguments");
    if (!c->have_gauge) return set_err(c, OV_ESTATE, "no gauge field");
    if (!c->net) return set_err(c, OV_ESTATE, "no network weights");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)npairs * 2 * c->g.Vh * 12 * 16;
    const double *dr = nullptr, *de = nullptr;
    FieldDesc fr, fe;
    OV_TRY(ws_field(c, WS_CG_R, P_F32, npairs, &fr));
    OV_TRY(ws_field(c, WS_CG_T, P_F32, npairs, &fe));
    OV_TRY(stage_in(c, 0, r, bytes, st, &dr));
    OV_CUDA(c, launch_pack(c->g, dr, fr, 0, st));
    OV_TRY(stage_in(c, 1, e, bytes, st, &de));
    OV_CUDA(c, launch_pack(c->g, de, fe, 0, st));
    OV_TRY(loss_grad(c, fr, fe, 0, npairs, loss, st));
    if (grad) {
        std::vector<float2> h(NET_PARAMS);
        OV_CUDA(c, cudaMemcpyAsync(h.data(), c->net->G, sizeof(float2) * NET_PARAMS, cudaMemcpyDeviceToHost, st));
        OV_CUDA(c, cudaStreamSynchronize(st));
        for (int i = 0; i < NET_PARAMS; ++i) {
            grad[2 * i] = h[i].x;
            grad[2 * i + 1] = h[i].y;
        }
    }
    return OV_OK;
}

int ov_net_train(ov_ctx* c, int nsolves, int steps, double lr, double mass, double* final_loss, void* stream)
{
    if (!c) return OV_EINVAL;
    if (nsolves < 1 || nsolves > 64 || steps < 0 || !(lr > 0)) return set_err(c, OV_EINVAL, "bad training arguments");
    if (!c->have_gauge || !c->have_poly) return set_err(c, OV_ESTATE, "training needs gauge field and sign polynomial");
    cudaStream_t st = (cudaStream_t)stream;
    OV_TRY(net_init(c));
    NetState* n = c->net;
    // ---- record (residual, iterate) pairs from deflated mixed-precision CG solves of random sources
    if (!n->pr.data) {
        n->cap = NET_MAXPAIRS;
        OV_TRY(field_alloc(c, P_F32, n->cap, &n->pr));
        OV_TRY(field_alloc(c, P_F32, n->cap, &n->px));
    }
    n->npairs = 0;
    FieldDesc b, xs32;
    OV_TRY(ws_field(c, WS_AUX1, P_F64, 1, &b));
    OV_TRY(ws_field(c, WS_NET_G, P_F32, 1, &xs32));
    const int was_trained = n->trained;
    n->trained = 0;
    for (int s = 0; s < nsolves && n->npairs < n->cap; ++s) {
        OV_CUDA(c, launch_fill_random(c->g, b, 9001ull + s, st));
        if (c->chiral) {  // chiral-sector solves need sources of definite chirality: alternate the sectors
            const double chi = (s & 1) ? -1.0 : 1.0;
            FieldDesc v2[2] = {b, b};
            double2 h2[2] = {make_double2(0.5, 0), make_double2(0.5 * chi, 0)};
            OV_TRY(lincomb(c, b, 2, v2, h2, nullptr, 2, nullptr, st));
        }
        const int first = n->npairs;
        n->recording = 1;
        FieldDesc bb, xx;
        OV_TRY(ws_field(c, WS_CG_B, P_F64, 1, &bb));
        OV_TRY(copy_field(c, b, bb, st));
        OV_TRY(ws_field(c, WS_CG_X, P_F64, 1, &xx));
        int r = cg_impl(c, bb, xx, mass, 1e-8, 400, 0, P_F32, nullptr, st);
        n->recording = 0;
        if (r != OV_OK && r != OV_ENOTCONV) return r;
        // e_k = x* - x_k (in place over the recorded iterates)
        OV_TRY(convert(c, xx, xs32, st));
        for (int k = first; k < n->npairs; ++k) {
            FieldDesc v[2] = {xs32, one(n->px, k)};
            double2 h[2] = {make_double2(1, 0), make_double2(-1, 0)};
            OV_TRY(lincomb(c, one(n->px, k), 2, v, h, nullptr, 0, nullptr, st));
        }
        // drop the last pair of the solve (converged: e ~ 0)
        if (n->npairs > first + 1) --n->npairs;
    }
    if (n->npairs < 2) return set_err(c, OV_ESTATE, "training: only %d pairs recorded", n->npairs);
    // ---- initialise: M = alpha * identity path (least-squares alpha), small deterministic noise elsewhere
    if (!was_trained) {
        std::vector<float2> w0(NET_PARAMS);
        unsigned long long z = 0x12345678ull;
        auto rnd = [&]() {
            z = z * 6364136223846793005ull + 1442695040888963407ull;
            return (float)((double)(z >> 11) / 9007199254740992.0 - 0.5);
        };
        for (auto& v : w0) v = make_float2(0.02f * rnd(), 0.02f * rnd());
        double num = 0, den = 0;
        for (int k = 0; k < n->npairs; ++k) {
            double* d = c->dscal + DSCAL_DOT;
            OV_TRY(dot(c, one(n->pr, k), one(n->px, k), (double2*)d, st));
            double2 re;
            OV_CUDA(c, cudaMemcpyAsync(&re, d, sizeof re, cudaMemcpyDeviceToHost, st));
            OV_TRY(norm2(c, one(n->pr, k), d, st));
            double2 rr;
            OV_CUDA(c, cudaMemcpyAsync(&rr, d, sizeof rr, cudaMemcpyDeviceToHost, st));
            OV_CUDA(c, cudaStreamSynchronize(st));
            double e2;
            OV_TRY(norm2(c, one(n->px, k), d, st));
            double2 ee;
            OV_CUDA(c, cudaMemcpyAsync(&ee, d, sizeof ee, cudaMemcpyDeviceToHost, st));
            OV_CUDA(c, cudaStreamSynchronize(st));
            e2 = ee.x > 0 ? ee.x : 1.0;
            num += re.x / e2;
            den += rr.x / e2;
        }
        const float alpha = (float)(den > 0 ? num / den : 1.0);
        for (int sa = 0; sa < 4; ++sa) {
            w0[(0 * NET_C + 0) * 16 + 5 * sa] = make_float2(1.f, 0.f);                   // layer 1, path 0, c=0
            w0[NET_W + (0 * 1 + 0) * NET_C * 16 + 5 * sa] = make_float2(alpha, 0.f);      // layer 2, path 0, c'=0
        }
        OV_CUDA(c, cudaMemcpyAsync(n->W, w0.data(), sizeof(float2) * NET_PARAMS, cudaMemcpyHostToDevice, st));
        OV_CUDA(c, cudaMemsetAsync(n->adam, 0, sizeof(float) * 4 * NET_PARAMS, st));
        n->adam_t = 0;
    }
    // ---- Adam over all recorded pairs
    double loss = 0;
    const float b1 = 0.9f, b2 = 0.999f;
    n->history.clear();
    for (int it = 0; it < steps; ++it) {
        OV_TRY(loss_grad(c, n->pr, n->px, 0, n->npairs, &loss, st));
        n->history.push_back(loss / n->npairs);
        ++n->adam_t;
        const float c1 = 1.f - powf(b1, (float)n->adam_t), c2 = 1.f - powf(b2, (float)n->adam_t);
        const float lr_t = (float)(lr * (it < steps / 2 ? 1.0 : 0.3));
        adam_kernel<<<(2 * NET_PARAMS + 255) / 256, 256, 0, st>>>(n->W, n->G, n->adam, n->adam + 2 * NET_PARAMS,
                                                                   NET_PARAMS, lr_t, b1, b2, 1e-8f, c1, c2,
                                                                   1.0f / (float)n->npairs);
        OV_CUDA(c, cudaGetLastError());
    }
    OV_TRY(loss_grad(c, n->pr, n->px, 0, n->npairs, &loss, st));  // also refreshes the adjoint weights
    if (final_loss) *final_loss = loss / n->npairs;
    n->history.push_back(loss / n->npairs);
    n->trained = 1;
    n->adj_valid = 1;
    return OV_OK;
}

int ov_net_pairs(const ov_ctx* c) { return c && c->net ? c->net->npairs : 0; }

int ov_net_loss_history(const ov_ctx* c, double* out, int cap)
{
    if (!c || cap < 0 || (cap > 0 && !out)) return -OV_EINVAL;
    if (!c->net) return 0;
    const auto& h = c->net->history;
    for (int i = 0; i < cap && i < (int)h.size(); ++i) out[i] = h[i];
    return (int)h.size();
}

}  // extern "C"
