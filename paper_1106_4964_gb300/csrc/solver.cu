// Solvers of the hot path, host logic over the library's kernels:
//  * estimate_lambda_max: Lanczos on H_w^2 for ||H_w|| (the spectral rescale Q = H_w / ||H_w||, Eq. 5);
//  * deflate_impl: Chebyshev-filtered subspace iteration with full FP64 Gram-Schmidt (CGS2): a block
//    filtered by T_K(Y(A)) of A = H_w^2 (Sec. V: Chebyshev acceleration, eigenvectors of T_n(H_w^2))
//    or of A = D^dag D, Rayleigh-Ritz with A every sweep, the filter's cut following the block's Ritz
//    values, then Rayleigh-Ritz with H_w for the signed eigenvalues of Eq. 7;
//  * cg_impl: deflated CG on D(m)^dag D(m) (Eq. 9) with mixed precision and reliable updates in FP64
//    or double-float, optionally with the one-sign chiral-sector inner operator (chiral_apply, api.cu)
//    and preconditioned by the learned network (flexible CG, net.cu).
// The paper uses implicitly restarted Arnoldi on the filtered operator; the operators here are
// Hermitian, and a filtered block iteration lets the filter interval adapt between sweeps.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <vector>

#include "ctx.h"

namespace ov {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------
// dense Hermitian eigensolver (cyclic Jacobi with complex rotations)
// A: n x n row-major Hermitian (destroyed).  ev ascending; Z[k*n + i] = component k of eigenvector i.
// ---------------------------------------------------------------------------
void herm_eig(int n, std::vector<cd>& A, std::vector<double>& ev, std::vector<cd>& Z)
{
    Z.assign((size_t)n * n, cd(0, 0));
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0, tot = 0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double a = std::norm(A[(size_t)p * n + q]);
                tot += a;
                if (p != q) off += a;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                cd apq = A[(size_t)p * n + q];
                double b = std::abs(apq);
                if (b == 0.0) continue;
                double al = A[(size_t)p * n + p].real(), be = A[(size_t)q * n + q].real();
                if (sweep > 3 && b < 1e-18 * (std::fabs(al) + std::fabs(be))) {
                    A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
                    continue;
                }
                cd u = apq / b, uc = std::conj(u);
                double zeta = (be - al) / (2.0 * b);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(zeta * zeta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    cd akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * uc * akq;
                    A[(size_t)k * n + q] = s * akp + c * uc * akq;
                }
                for (int k = 0; k < n; ++k) {
                    cd apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * u * aqk;
                    A[(size_t)q * n + k] = s * apk + c * u * aqk;
                }
                A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
                A[(size_t)p * n + p] = al - t * b;
                A[(size_t)q * n + q] = be + t * b;
                for (int k = 0; k < n; ++k) {
                    cd zkp = Z[(size_t)k * n + p], zkq = Z[(size_t)k * n + q];
                    Z[(size_t)k * n + p] = c * zkp - s * uc * zkq;
                    Z[(size_t)k * n + q] = s * zkp + c * uc * zkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(),
              [&](int a, int b) { return A[(size_t)a * n + a].real() < A[(size_t)b * n + b].real(); });
    ev.resize(n);
    std::vector<cd> Zs((size_t)n * n);
    for (int i = 0; i < n; ++i) {
        ev[i] = A[(size_t)idx[i] * n + idx[i]].real();
        for (int k = 0; k < n; ++k) Zs[(size_t)k * n + i] = Z[(size_t)k * n + idx[i]];
    }
    Z.swap(Zs);
}

namespace {

FieldDesc sub(const FieldDesc& f, int i, int n = 1)
{
    FieldDesc s = f;
    s.nrhs = n;
    s.data = f.data + (size_t)i * f.rhs_bytes();
    s.norm = f.norm ? f.norm + (size_t)i * 2 * f.Vh : nullptr;
    return s;
}

int to_host(ov_ctx* c, const void* d, void* h, size_t bytes, cudaStream_t st)
{
    OV_CUDA(c, cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    return OV_OK;
}

int to_dev(ov_ctx* c, const void* h, void* d, size_t bytes, cudaStream_t st)
{
    OV_CUDA(c, cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st));
    return OV_OK;
}

// h[i][r] = basis_i^dag w_r for i < n  (device result in c->dscal as double2 [n][R])
int block_dots(ov_ctx* c, const FieldDesc& basis, int n, const FieldDesc& w, cudaStream_t st)
{
    const int nblk = reduce_blocks(c->g);
    const int nparts = nblk * proj_groups(w.nrhs);
    const size_t ncoef = (size_t)n * w.nrhs;
    if (ncoef * 2 > (size_t)DSCAL_COEF) return set_err(c, OV_EINVAL, "block of %zu coefficients too large", ncoef);
    OV_TRY(ensure_partials(c, nparts * ncoef * sizeof(double2)));
    OV_CUDA(c, launch_proj_dots(c->g, basis, n, w, (double2*)c->partials, nblk, st));
    OV_CUDA(c, launch_proj_finalize((double2*)c->partials, nparts, (int)ncoef, (double2*)c->dscal, st));
    return OV_OK;
}

// w_r -= sum_i basis_i coef[i][r], coef (device double2 [n][R]) in c->dscal
int block_sub(ov_ctx* c, const FieldDesc& basis, int n, const FieldDesc& w, cudaStream_t st)
{
    FieldDesc none{};
    OV_CUDA(c, launch_proj_update(c->g, basis, n, (const double2*)c->dscal, nullptr, w, w, none, st));
    return OV_OK;
}

// out_j = sum_i basis_i Y[i][j] for j < k (Y host, n x k, ld = ldy), through the zero field `zero` (16 rhs)
int rotate(ov_ctx* c, const FieldDesc& basis, int n, const std::vector<cd>& Y, int ldy, int k, const FieldDesc& out,
           const FieldDesc& zero, cudaStream_t st)
{
    for (int j0 = 0; j0 < k; j0 += 16) {
        const int nr = std::min(16, k - j0);
        std::vector<double2> coef((size_t)n * nr);
        for (int i = 0; i < n; ++i)
            for (int r = 0; r < nr; ++r) {
                cd y = Y[(size_t)i * ldy + j0 + r];
                coef[(size_t)i * nr + r] = make_double2(-y.real(), -y.imag());
            }
        if (coef.size() * 2 > (size_t)DSCAL_COEF) return set_err(c, OV_EINVAL, "rotation block too large");
        OV_TRY(to_dev(c, coef.data(), c->dscal, coef.size() * sizeof(double2), st));
        FieldDesc z = sub(zero, 0, nr), o = sub(out, j0, nr);
        FieldDesc none{};
        OV_CUDA(c, launch_proj_update(c->g, basis, n, (const double2*)c->dscal, nullptr, z, o, none, st));
        OV_CUDA(c, cudaStreamSynchronize(st));  // c->dscal is reused by the next block
    }
    return OV_OK;
}

double host_norm(ov_ctx* c, const FieldDesc& x, cudaStream_t st, int* status)
{
    *status = norm2(c, x, c->dscal + DSCAL_TMP, st);
    if (*status != OV_OK) return 0;
    double2 v;
    *status = to_host(c, c->dscal + DSCAL_TMP, &v, sizeof v, st);
    return std::sqrt(v.x);
}

int scale_into(ov_ctx* c, const FieldDesc& in, const FieldDesc& out, double s, cudaStream_t st)
{
    double2 h = make_double2(s, 0);
    return lincomb(c, out, 1, &in, &h, nullptr, 0, nullptr, st);
}

using OpFn = std::function<int(const FieldDesc&, const FieldDesc&)>;

// Chebyshev filter: out = T_K(Y) in, Y = (2 A - (a+b)) / (b-a), three-term recurrence
// The recurrence runs in the precision of the work fields tmp[0..3] (A acts on
// fields of that precision); in and out are converted once if they differ.
// K = 0 gives the plain spectral flip F = b - A (largest of F = smallest of A).
int cheb_filter(ov_ctx* c, const OpFn& A, int K, double a, double b, const FieldDesc& in, const FieldDesc& out,
                FieldDesc tmp[4], cudaStream_t st)
{
    const bool conv = tmp[0].prec != in.prec;
    FieldDesc q = tmp[0], y_prev = tmp[1], y_cur = tmp[2];
    FieldDesc x0 = in;
    if (conv) {
        x0 = tmp[3];
        OV_TRY(convert(c, in, x0, st));
    }
    FieldDesc last;
    if (K == 0) {
        OV_TRY(A(x0, q));
        last = conv ? y_cur : out;
        FieldDesc xs[2] = {x0, q};
        double2 h[2] = {make_double2(b, 0), make_double2(-1, 0)};
        OV_TRY(lincomb(c, last, 2, xs, h, nullptr, 0, nullptr, st));
    } else {
        const double s1 = 2.0 / (b - a), s0 = -(a + b) / (b - a);
        OV_TRY(A(x0, q));  // y1 = Y y0
        if (conv)
            y_prev = x0;  // the converted input is a work field of its own
        else
            OV_TRY(copy_field(c, x0, y_prev, st));
        last = (K == 1 && !conv) ? out : y_cur;
        {
            FieldDesc xs[2] = {q, x0};
            double2 h[2] = {make_double2(s1, 0), make_double2(s0, 0)};
            OV_TRY(lincomb(c, last, 2, xs, h, nullptr, 0, nullptr, st));
        }
        for (int j = 1; j < K; ++j) {
            OV_TRY(A(y_cur, q));
            FieldDesc dst = (j == K - 1 && !conv) ? out : y_prev;  // y_{j+1} overwrites y_{j-1}
            FieldDesc xs[3] = {q, y_cur, y_prev};
            double2 h[3] = {make_double2(2 * s1, 0), make_double2(2 * s0, 0), make_double2(-1, 0)};
            OV_TRY(lincomb(c, dst, 3, xs, h, nullptr, 0, nullptr, st));
            last = dst;
            std::swap(y_prev, y_cur);
        }
    }
    if (conv) OV_TRY(convert(c, last, out, st));
    return OV_OK;
}

// Full CGS2 of w against basis[0..n): returns the coefficient sum in h (host)
int cgs2(ov_ctx* c, const FieldDesc& basis, int n, const FieldDesc& w, std::vector<cd>& h, cudaStream_t st)
{
    h.assign(n, cd(0, 0));
    for (int pass = 0; pass < 2; ++pass) {
        OV_TRY(block_dots(c, basis, n, w, st));
        std::vector<double2> hh(n);
        OV_TRY(to_host(c, c->dscal, hh.data(), n * sizeof(double2), st));
        for (int i = 0; i < n; ++i) h[i] += cd(hh[i].x, hh[i].y);
        OV_TRY(block_sub(c, basis, n, w, st));
    }
    return OV_OK;
}

// m-step Lanczos with full reorthogonalisation on a Hermitian operator; returns the Ritz values
int plain_lanczos(ov_ctx* c, const OpFn& A, int m, const FieldDesc& basis, const FieldDesc& w, unsigned long long seed,
                  std::vector<double>& ritz, cudaStream_t st)
{
    int status = OV_OK;
    OV_CUDA(c, launch_fill_random(c->g, sub(basis, 0), seed, st));
    double nr = host_norm(c, sub(basis, 0), st, &status);
    OV_TRY(status);
    OV_TRY(scale_into(c, sub(basis, 0), sub(basis, 0), 1.0 / nr, st));
    std::vector<cd> T((size_t)m * m, cd(0, 0));
    int mm = m;
    for (int j = 0; j < m; ++j) {
        OV_TRY(A(sub(basis, j), w));
        std::vector<cd> h;
        OV_TRY(cgs2(c, basis, j + 1, w, h, st));
        for (int i = 0; i <= j; ++i) {
            T[(size_t)i * m + j] = h[i];
            T[(size_t)j * m + i] = std::conj(h[i]);
        }
        double beta = host_norm(c, w, st, &status);
        OV_TRY(status);
        if (j + 1 < m) {
            if (beta < 1e-12 * std::abs(T[(size_t)j * m + j]) + 1e-300) {
                mm = j + 1;
                break;
            }
            OV_TRY(scale_into(c, w, sub(basis, j + 1), 1.0 / beta, st));
        }
    }
    std::vector<cd> Tm((size_t)mm * mm);
    for (int i = 0; i < mm; ++i)
        for (int j = 0; j < mm; ++j) Tm[(size_t)i * mm + j] = T[(size_t)i * m + j];
    std::vector<cd> Z;
    herm_eig(mm, Tm, ritz, Z);
    return OV_OK;
}

}  // namespace

int estimate_lambda_max(ov_ctx* c, int steps, double* lmax, cudaStream_t st)
{
    const long long N = 24LL * c->g.Vh;  // complex dimension 12 V
    int m = (int)std::min<long long>(steps, N);
    FieldDesc basis, w, t;
    OV_TRY(field_alloc(c, P_F64, m, &basis));
    int s = ws_field(c, WS_LZ_W, P_F64, 1, &w);
    if (s == OV_OK) s = ws_field(c, WS_LZ_T, P_F64, 1, &t);
    std::vector<double> ritz;
    if (s == OV_OK) {
        OpFn H2 = [&](const FieldDesc& in, const FieldDesc& out) -> int {
            OV_TRY(dslash_apply(c, in, t, 4.0 - c->rho, -0.5, 1, 0, 0, nullptr, nullptr, st));
            return dslash_apply(c, t, out, 4.0 - c->rho, -0.5, 1, 0, 0, nullptr, nullptr, st);
        };
        s = plain_lanczos(c, H2, m, basis, w, 12345ull, ritz, st);
    }
    cudaStreamSynchronize(st);
    field_free(c, &basis);
    OV_TRY(s);
    *lmax = std::sqrt(std::max(0.0, ritz.back()));
    return OV_OK;
}

namespace {

// v <- P_chi v = (v + chi gamma5 v) / 2 (chi = +-1); nothing for chi = 0
int project_chiral(ov_ctx* c, const FieldDesc& v, int chi, cudaStream_t st)
{
    if (!chi) return OV_OK;
    FieldDesc xs[2] = {v, v};
    double2 h[2] = {make_double2(0.5, 0), make_double2(0.5 * chi, 0)};
    return lincomb(c, v, 2, xs, h, nullptr, 2, nullptr, st);
}

struct LanczosWork {
    FieldDesc basis, rot, zero, w, wb, tmp[4];  // wb: FP64 batch of the filter (FB right-hand sides)
};

// Chebyshev-filtered subspace iteration for the nev smallest eigenpairs of the Hermitian A on
// the chirality-chi subspace (chi = 0: whole space; +-1: gamma5 = chi, enforced after every
// operator application).  A block of nb orthonormal FP64 vectors is filtered with T_K(Y(A)) on
// [acut, bmax] (work-precision fields), re-orthonormalised by CGS2 and Rayleigh-Ritz-projected
// with A.  The cut starts at an upper bound of the eigenvalue of index nb from a short
// unfiltered Lanczos run (Ritz values bound the eigenvalues of the same index from above) and
// then follows the largest Ritz value of the block, also an upper bound of that eigenvalue
// (Courant-Fischer), so the filter sharpens as the block converges.  Leading Ritz vectors whose
// A-residual is small enough are locked (no longer filtered).  Finally the nev leading vectors
// are rotated by Rayleigh-Ritz with R and accepted when max_i |R eta_i - lam_i eta_i| <=
// tol * rscale.  sq: A = R^2 (an R-residual e shows as about 2 |lam| e in A).  refine(): switch
// A and Awork to the accurate precision (false when they already are); called when the final
// check fails.  Vectors go to `out` (nev fields), values (sorted by |lam|) to vals.
int chfsi(ov_ctx* c, const OpFn& A, const OpFn& Awork, const OpFn& R, int K, double bmax, int nev, int nb,
          double tol, double rscale, bool sq, int chi, unsigned long long seed, LanczosWork& W,
          const std::function<bool()>& refine, std::vector<double>& vals, const FieldDesc& out, double* maxres_out,
          cudaStream_t st)
{
    int status = OV_OK;
    const FieldDesc& V = W.basis;
    OpFn Ac = [&](const FieldDesc& in, const FieldDesc& o) -> int {
        OV_TRY(A(in, o));
        return project_chiral(c, o, chi, st);
    };
    OpFn AcW = [&](const FieldDesc& in, const FieldDesc& o) -> int {
        OV_TRY(Awork(in, o));
        return project_chiral(c, o, chi, st);
    };
    // normalised w -> V_j after CGS2 against V[0..j); a random vector replaces a vanishing one
    auto orth_into = [&](int j, unsigned long long s) -> int {
        for (int attempt = 0; attempt < 3; ++attempt) {
            std::vector<cd> h;
            if (j > 0) OV_TRY(cgs2(c, V, j, W.w, h, st));
            const double nr = host_norm(c, W.w, st, &status);
            OV_TRY(status);
            if (nr > 1e-200) return scale_into(c, W.w, sub(V, j), 1.0 / nr, st);
            OV_CUDA(c, launch_fill_random(c->g, W.w, s + 7919ull * (attempt + 1), st));
            OV_TRY(project_chiral(c, W.w, chi, st));
        }
        return set_err(c, OV_ENOTCONV, "eigensolver: block vector %d vanished", j);
    };

    // cut: upper bound of lambda_{nb} from an unfiltered Lanczos run
    double acut;
    {
        const int m0 = std::min(V.nrhs - 1, nb + 40);
        OV_CUDA(c, launch_fill_random(c->g, sub(V, 0), seed + 101, st));
        OV_TRY(project_chiral(c, sub(V, 0), chi, st));
        double nr = host_norm(c, sub(V, 0), st, &status);
        OV_TRY(status);
        OV_TRY(scale_into(c, sub(V, 0), sub(V, 0), 1.0 / nr, st));
        std::vector<cd> T((size_t)m0 * m0, cd(0, 0));
        int mm = m0;
        for (int j = 0; j < m0; ++j) {
            OV_TRY(Ac(sub(V, j), W.w));
            std::vector<cd> h;
            OV_TRY(cgs2(c, V, j + 1, W.w, h, st));
            for (int i = 0; i <= j; ++i) {
                T[(size_t)i * m0 + j] = h[i];
                T[(size_t)j * m0 + i] = std::conj(h[i]);
            }
            const double beta = host_norm(c, W.w, st, &status);
            OV_TRY(status);
            if (j + 1 < m0) {
                if (beta < 1e-12 * std::abs(T[(size_t)j * m0 + j]) + 1e-300) {
                    mm = j + 1;
                    break;
                }
                OV_TRY(scale_into(c, W.w, sub(V, j + 1), 1.0 / beta, st));
            }
        }
        std::vector<cd> Tm((size_t)mm * mm), Zt;
        for (int i = 0; i < mm; ++i)
            for (int j = 0; j < mm; ++j) Tm[(size_t)i * mm + j] = T[(size_t)i * m0 + j];
        std::vector<double> ritz0;
        herm_eig(mm, Tm, ritz0, Zt);
        acut = ritz0[std::min((int)ritz0.size() - 1, nb - 1)];
        if (!(acut < bmax)) acut = 0.5 * bmax;
    }
    // random orthonormal block
    for (int j = 0; j < nb; ++j) {
        OV_CUDA(c, launch_fill_random(c->g, W.w, seed + 1000003ull * (j + 1), st));
        OV_TRY(project_chiral(c, W.w, chi, st));
        OV_TRY(orth_into(j, seed + j));
    }

    // |op(B_{w0+q}) - lam[q] B_{w0+q}| for the FB vectors of B from w0 (one multi-RHS application),
    // into rwin[q]
    const int FB = W.wb.nrhs;
    std::vector<double> rwin(FB);
    auto residual_window = [&](const OpFn& op, const FieldDesc& B, int w0, const double* lam, int n) -> int {
        OV_TRY(op(sub(B, w0, n), W.wb));
        std::vector<double2> co(2 * n);
        for (int q = 0; q < n; ++q) {
            co[q] = make_double2(1, 0);
            co[n + q] = make_double2(-lam[q], 0);
        }
        double2* dco = (double2*)(c->dscal + DSCAL_CGCO);
        double* dnr = c->dscal + DSCAL_NORM;
        OV_TRY(to_dev(c, co.data(), dco, co.size() * sizeof(double2), st));
        FieldDesc xs[2] = {W.wb, sub(B, w0, n)};
        OV_TRY(lincomb(c, W.wb, 2, xs, nullptr, dco, 0, dnr, st));
        std::vector<double> n2(n);
        OV_TRY(to_host(c, dnr, n2.data(), n * sizeof(double), st));
        for (int q = 0; q < n; ++q) rwin[q] = std::sqrt(std::max(0.0, n2[q]));
        return OV_OK;
    };
    std::vector<double> theta(nb, 0.0), res(nb, 1e300);
    int nlock = 0;
    double tscale = 1.0;  // tightens the locking threshold when the final R check fails
    auto tolA = [&](double th) {
        return tscale * (sq ? tol * rscale * std::sqrt(std::max(th, 0.0)) : 0.5 * tol * rscale);
    };
    double maxres = 1e300;
    for (int it = 0; it < 300; ++it) {
        // degree: even (T_K > 0 below the cut) and capped so that T_K(0) stays within what the work
        // precision resolves (1e12 FP64, 1e10 double-float, 1e4 FP32)
        // largest amplification among the vectors still filtered: at the smallest unlocked Ritz value
        const double lo_th = it == 0 ? 0.0 : std::max(0.0, std::min(theta[nlock], acut));
        const double y0 = (bmax + acut - 2.0 * lo_th) / (bmax - acut);
        const double limit = W.tmp[0].prec == P_F64 ? 1e12 : (W.tmp[0].prec == P_DF64 ? 1e10 : 1e4);
        const int kmax = (int)std::floor(std::acosh(limit) / std::acosh(y0));
        const int Keff = std::max(2, std::min(K, kmax)) & ~1;
        // The unlocked vectors are filtered FB at a time as one multi-RHS field (the multi-RHS
        // operator costs less per vector than FB single ones), a window of exactly FB vectors so that
        // every batch reuses the same work fields (the last window reaches back over vectors already
        // done, whose filtered copies are dropped).  The batch is orthogonalised against V[0, j0) by
        // a block CGS2 (one pass over V per pass for all FB vectors), then each vector against the
        // batch vectors placed before it.
        for (int j0 = nlock; j0 < nb; j0 += FB) {
            const int w0 = std::max(0, std::min(j0, nb - FB));
            OV_TRY(cheb_filter(c, AcW, Keff, acut, bmax, sub(V, w0, FB), W.wb, W.tmp, st));
            OV_TRY(project_chiral(c, W.wb, chi, st));
            if (j0 > 0)
                for (int pass = 0; pass < 2; ++pass) {
                    OV_TRY(block_dots(c, V, j0, W.wb, st));
                    OV_TRY(block_sub(c, V, j0, W.wb, st));
                }
            for (int j = j0; j < std::min(j0 + FB, nb); ++j) {
                OV_TRY(copy_field(c, sub(W.wb, j - w0), W.w, st));
                std::vector<cd> h;
                if (j > j0) OV_TRY(cgs2(c, sub(V, j0, j - j0), j - j0, W.w, h, st));
                const double nr = host_norm(c, W.w, st, &status);
                OV_TRY(status);
                if (nr > 1e-200)
                    OV_TRY(scale_into(c, W.w, sub(V, j), 1.0 / nr, st));
                else
                    OV_TRY(orth_into(j, seed + 31ull * it + j));  // vanished: a random vector in its place
            }
        }
        // Rayleigh-Ritz with A over the block (locked vectors keep their Ritz values); the columns
        // A V_j in windows of FB vectors, like the filter
        std::vector<cd> G((size_t)nb * nb, cd(0, 0));
        for (int j0 = nlock; j0 < nb; j0 += FB) {
            const int w0 = std::max(0, std::min(j0, nb - FB));
            OV_TRY(Ac(sub(V, w0, FB), W.wb));
            OV_TRY(block_dots(c, V, nb, W.wb, st));
            std::vector<double2> hh((size_t)nb * FB);
            OV_TRY(to_host(c, c->dscal, hh.data(), hh.size() * sizeof(double2), st));
            for (int j = j0; j < std::min(j0 + FB, nb); ++j)
                for (int i = 0; i < nb; ++i) {
                    const double2 v = hh[(size_t)i * FB + (j - w0)];
                    G[(size_t)i * nb + j] = cd(v.x, v.y);
                }
        }
        for (int i = 0; i < nb; ++i) {
            if (i < nlock) {
                G[(size_t)i * nb + i] = theta[i];
                for (int j = nlock; j < nb; ++j) G[(size_t)j * nb + i] = std::conj(G[(size_t)i * nb + j]);
                continue;
            }
            for (int j = i; j < nb; ++j) {
                const cd a = 0.5 * (G[(size_t)i * nb + j] + std::conj(G[(size_t)j * nb + i]));
                G[(size_t)i * nb + j] = a;
                G[(size_t)j * nb + i] = std::conj(a);
            }
        }
        std::vector<double> th;
        std::vector<cd> S;
        herm_eig(nb, G, th, S);
        OV_TRY(rotate(c, V, nb, S, nb, nb, W.rot, W.zero, st));
        OV_CUDA(c, cudaMemcpyAsync(V.data, W.rot.data, V.rhs_bytes() * nb, cudaMemcpyDeviceToDevice, st));
        theta = th;
        // Lock the leading Ritz vectors whose A-residual is small enough: residuals are recomputed
        // every sweep (the Rayleigh-Ritz step may reorder the block) and as far as the locked run
        // extends, past nev when it can (a few block vectors stay unlocked as a buffer).
        nlock = 0;
        const int jmax = std::max(nev, nb - 4);
        bool ended = false;
        for (int j0 = 0; j0 < jmax && !ended; j0 += FB) {
            const int w0 = std::max(0, std::min(j0, nb - FB));
            OV_TRY(residual_window(Ac, V, w0, theta.data() + w0, FB));
            for (int j = j0; j < std::min(j0 + FB, jmax); ++j) {
                res[j] = rwin[j - w0];
                if (j == nlock && res[j] <= tolA(theta[j])) ++nlock;
                if (j >= nev - 1 && j >= nlock) {  // the locked run ended
                    ended = true;
                    break;
                }
            }
        }
        if (verbose())
            fprintf(stderr, "[ov] chfsi chi=%d it %d: cut %.4e, degree %d, locked %d (want %d), res[nev-1] %.3e\n", chi,
                    it, acut, Keff, nlock, nev, res[nev - 1]);
        if (nlock >= nev) {
            // Rayleigh-Ritz with R over every locked vector.  The locked set holds all A-eigenvectors
            // below its largest Ritz value, so it is R-invariant except where a +-lambda pair of
            // R^2 = A straddles its edge (a mixture of the two partners); such Ritz pairs show a large
            // R-residual.  The accepted set is the smallest-|lambda| prefix of good pairs, so that no
            // mode below the largest accepted |lambda| is left out of the deflation.
            const int nr = nlock;
            std::vector<cd> M((size_t)nr * nr);
            for (int j0 = 0; j0 < nr; j0 += FB) {
                const int w0 = std::max(0, std::min(j0, nb - FB));
                OV_TRY(R(sub(V, w0, FB), W.wb));
                OV_TRY(block_dots(c, V, nr, W.wb, st));
                std::vector<double2> hh((size_t)nr * FB);
                OV_TRY(to_host(c, c->dscal, hh.data(), hh.size() * sizeof(double2), st));
                for (int j = j0; j < std::min(j0 + FB, nr); ++j)
                    for (int i = 0; i < nr; ++i) {
                        const double2 v = hh[(size_t)i * FB + (j - w0)];
                        M[(size_t)i * nr + j] = cd(v.x, v.y);
                    }
            }
            for (int i = 0; i < nr; ++i)
                for (int j = i; j < nr; ++j) {
                    const cd a = 0.5 * (M[(size_t)i * nr + j] + std::conj(M[(size_t)j * nr + i]));
                    M[(size_t)i * nr + j] = a;
                    M[(size_t)j * nr + i] = std::conj(a);
                }
            std::vector<double> lam;
            std::vector<cd> Sr;
            herm_eig(nr, M, lam, Sr);
            std::vector<int> o(nr);
            for (int i = 0; i < nr; ++i) o[i] = i;
            std::sort(o.begin(), o.end(), [&](int a, int b) { return std::fabs(lam[a]) < std::fabs(lam[b]); });
            std::vector<cd> So((size_t)nr * nr);
            std::vector<double> lo(nr);
            for (int j = 0; j < nr; ++j) {
                lo[j] = lam[o[j]];
                for (int i = 0; i < nr; ++i) So[(size_t)i * nr + j] = Sr[(size_t)i * nr + o[j]];
            }
            FieldDesc eta = sub(W.rot, 0, nr);
            OV_TRY(rotate(c, V, nr, So, nr, nr, eta, W.zero, st));
            int good = 0;
            maxres = 0;
            bool bad = false;
            for (int j0 = 0; j0 < nr && !bad; j0 += FB) {
                // windows inside W.rot (nb vectors; past nr it holds earlier, finite rotations)
                const int w0 = std::max(0, std::min(j0, nb - FB));
                std::vector<double> lw(FB, 0.0);
                for (int q = 0; q < FB; ++q)
                    if (w0 + q < nr) lw[q] = lo[w0 + q];
                OV_TRY(residual_window(R, W.rot, w0, lw.data(), FB));
                for (int j = j0; j < std::min(j0 + FB, nr); ++j) {
                    const double r = rwin[j - w0] / rscale;
                    if (r > tol) {
                        bad = true;
                        break;
                    }
                    maxres = std::max(maxres, r);
                    ++good;
                }
            }
            if (verbose())
                fprintf(stderr, "[ov] chfsi chi=%d: Rayleigh-Ritz over %d locked vectors, %d good (want %d)\n", chi, nr,
                        good, nev);
            if (good >= nev) {
                OV_CUDA(c, cudaMemcpyAsync(out.data, eta.data, eta.rhs_bytes() * nev, cudaMemcpyDeviceToDevice, st));
                OV_CUDA(c, cudaStreamSynchronize(st));
                vals.assign(lo.begin(), lo.begin() + nev);
                *maxres_out = maxres;
                return OV_OK;
            }
            if (refine()) {
                // the work precision's own eigenvectors differ from the accurate ones by its rounding
                // over the gaps; in a dense cluster that mixes many of them: continue accurately
                if (verbose()) fprintf(stderr, "[ov] chfsi chi=%d: continuing with the accurate operator\n", chi);
            }
            // In a dense cluster an A-residual near the locking threshold still mixes neighbouring
            // modes by more than the R criterion allows: tighten it (the accurate operator resolves it)
            tscale = std::max(tscale * 0.1, 1e-6);
        }
        if (theta[nb - 1] > theta[nev - 1] && theta[nb - 1] < acut) acut = theta[nb - 1];
    }
    *maxres_out = maxres;
    return set_err(c, OV_ENOTCONV, "eigensolver: not converged (max eigen-residual %.3e > tol %.3e)", maxres, tol);
}

int store_eigs(ov_ctx* c, int which, const FieldDesc& vecs, const std::vector<int>& pick,
               const std::vector<double>& vals, cudaStream_t st)
{
    EigSet& E = c->eig[which];
    graphs_clear(c);
    eig_clear(c, E);
    const int nev = (int)pick.size();
    OV_TRY(field_alloc(c, P_F64, nev, &E.vec[P_F64]));
    std::vector<double> sg(nev);
    for (int i = 0; i < nev; ++i) {
        OV_CUDA(c, cudaMemcpyAsync(sub(E.vec[P_F64], i).data, sub(vecs, pick[i]).data, vecs.rhs_bytes(),
                                   cudaMemcpyDeviceToDevice, st));
        E.vals.push_back(vals[pick[i]]);
        sg[i] = vals[pick[i]] > 0 ? 1.0 : (vals[pick[i]] < 0 ? -1.0 : 0.0);
    }
    void* p = nullptr;
    OV_TRY(dev_alloc(c, &p, sizeof(double) * nev));
    E.d_sign = (double*)p;
    OV_CUDA(c, cudaMemcpyAsync(E.d_sign, sg.data(), sizeof(double) * nev, cudaMemcpyHostToDevice, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    E.nev = nev;
    return OV_OK;
}

}  // namespace

// which = 0: nev smallest-|lambda| eigenpairs of H_w (subspace iteration with the filter T_100(Y(H_w^2)),
//            Rayleigh-Ritz with H_w).
// which = 1: nev smallest eigenpairs of D(0)^dag D(0).  It commutes with gamma5 and its eigenvalues
//            are doubly degenerate across the two chiral sectors (d and d* of D share |d|^2), which a
//            single-vector Krylov method cannot resolve, so each sector is solved on its own (the chiral
//            structure Sec. V uses) and the lowest nev of the union are kept.
int deflate_impl(ov_ctx* c, int which, int nev, double tol, cudaStream_t st)
{
    const long long N = 24LL * c->g.Vh;  // complex dimension 12 V
    const int nsec = which == 0 ? 1 : 2;
    const long long dim = which == 0 ? N : N / 2;
    const int ns = which == 0 ? nev : std::min<long long>(nev / 2 + 4, nev);
    if (ns >= dim / 2) return set_err(c, OV_EINVAL, "nev = %d too large for a lattice of dimension %lld", nev, N);
    // block of the filtered subspace iteration, and the unfiltered Lanczos run that sets the first cut
    const int nb = (int)std::min<long long>(ns + std::max(16, (3 * ns) / 4), dim / 2);
    const int m0 = (int)std::min<long long>(nb + 40, dim - 1);
    // operator precision: FP64 when the eigen-residual target needs it; an FP32 filter (FP64
    // Gram-Schmidt and Rayleigh-Ritz) when tol >= 1e-7, or as set by ov_set_option("eig_prec")
    const int oprec = c->eig_prec >= 0 ? c->eig_prec : (tol >= 1e-5 ? P_F32 : c->hi_prec);

    LanczosWork W{};
    FieldDesc outv{};
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        field_free(c, &W.basis);
        field_free(c, &W.rot);
        field_free(c, &outv);
    };
#define DF_TRY(x)           \
    do {                    \
        int s__ = (x);      \
        if (s__ != OV_OK) { \
            cleanup();      \
            return s__;     \
        }                   \
    } while (0)
    DF_TRY(field_alloc(c, P_F64, std::max(nb, m0 + 1), &W.basis));
    DF_TRY(field_alloc(c, P_F64, nb, &W.rot));
    DF_TRY(field_alloc(c, P_F64, nsec * ns, &outv));
    DF_TRY(ws_field(c, WS_AUX1, P_F64, 16, &W.zero));
    DF_TRY(ws_field(c, WS_LZ_W, P_F64, 1, &W.w));
    const int FB = std::min(12, nb);  // filter batch: as many right-hand sides as a propagator solve
    DF_TRY(ws_field(c, WS_LZ_WB, P_F64, FB, &W.wb));
    // windows of FB vectors may reach past the rotated vectors of W.rot: keep them finite
    OV_CUDA(c, cudaMemsetAsync(W.rot.data, 0, W.rot.rhs_bytes() * nb, st));
    OV_CUDA(c, cudaMemsetAsync(W.zero.data, 0, W.zero.rhs_bytes() * 16, st));
    // Operator precision `cur`: the filter temporaries (slots of their own: the Clenshaw buffers
    // are used inside D^dag D) and, below FP64, conversion fields (in, out, middle).
    int cur = oprec;
    auto prepare = [&](int p) -> int {
        OV_TRY(ws_field(c, WS_LZ_F0, p, FB, &W.tmp[0]));
        OV_TRY(ws_field(c, WS_LZ_F1, p, FB, &W.tmp[1]));
        OV_TRY(ws_field(c, WS_LZ_F2, p, FB, &W.tmp[2]));
        OV_TRY(ws_field(c, WS_LZ_F3, p, FB, &W.tmp[3]));
        return OV_OK;
    };
    DF_TRY(prepare(oprec));
    // continue in the accurate precision when the work precision's eigenvectors are not good enough
    std::function<bool()> refine = [&]() -> bool {
        const int hi = c->hi_prec;
        if (cur == hi || cur == P_F64 || prepare(hi) != OV_OK) return false;
        cur = hi;
        return true;
    };

    OpFn A, Awork, R;
    double bmax, rscale;
    int K;
    if (which == 0) {
        Awork = [&](const FieldDesc& in, const FieldDesc& out) -> int {  // the filter's batch
            FieldDesc tmid;
            OV_TRY(ws_field(c, WS_LZ_T, cur, in.nrhs, &tmid));
            OV_TRY(dslash_apply(c, in, tmid, 4.0 - c->rho, -0.5, 1, 0, 0, nullptr, nullptr, st));
            return dslash_apply(c, tmid, out, 4.0 - c->rho, -0.5, 1, 0, 0, nullptr, nullptr, st);
        };
        A = [&](const FieldDesc& in, const FieldDesc& out) -> int {  // one vector or a window of FB
            FieldDesc t;
            OV_TRY(ws_field(c, WS_LZ_T, cur, in.nrhs, &t));
            if (cur == P_F64) {
                OV_TRY(dslash_apply(c, in, t, 4.0 - c->rho, -0.5, 1, 0, 0, nullptr, nullptr, st));
                return dslash_apply(c, t, out, 4.0 - c->rho, -0.5, 1, 0, 0, nullptr, nullptr, st);
            }
            FieldDesc a, b;
            OV_TRY(ws_field(c, WS_CG_RS, cur, in.nrhs, &a));
            OV_TRY(ws_field(c, WS_CG_QS, cur, in.nrhs, &b));
            OV_TRY(convert(c, in, a, st));
            OV_TRY(dslash_apply(c, a, t, 4.0 - c->rho, -0.5, 1, 0, 0, nullptr, nullptr, st));
            OV_TRY(dslash_apply(c, t, b, 4.0 - c->rho, -0.5, 1, 0, 0, nullptr, nullptr, st));
            return convert(c, b, out, st);
        };
        R = [&](const FieldDesc& in, const FieldDesc& out) -> int {
            return dslash_apply(c, in, out, 4.0 - c->rho, -0.5, 1, 0, 0, nullptr, nullptr, st);
        };
        double lm = c->lmax;
        if (!(lm > 0)) {
            DF_TRY(estimate_lambda_max(c, 50, &lm, st));
            lm *= 1.01;
        }
        bmax = lm * lm;
        rscale = lm;
        K = c->filter_hw;
    } else {
        // D^dag D, or with the "chiral" option its one-sign form on the sector being solved
        // (coefficients [3][R]: at dchi for one vector, at dchi + 8 for the filter's batch)
        const double2* dchi = (const double2*)(c->dscal + DSCAL_CHCO);
        Awork = [&, dchi](const FieldDesc& in, const FieldDesc& out) -> int {
            const double2* dc = in.nrhs == 1 ? dchi : dchi + 8;
            return c->chiral ? chiral_apply(c, in, out, 0.0, dc, st) : normal_apply(c, in, out, 0.0, st);
        };
        A = [&](const FieldDesc& in, const FieldDesc& out) -> int {  // one vector or a window of FB
            if (cur == P_F64) return Awork(in, out);
            FieldDesc a, b;
            OV_TRY(ws_field(c, WS_CG_RS, cur, in.nrhs, &a));
            OV_TRY(ws_field(c, WS_CG_QS, cur, in.nrhs, &b));
            OV_TRY(convert(c, in, a, st));
            OV_TRY(Awork(a, b));
            return convert(c, b, out, st);
        };
        R = A;
        bmax = 4.0 * c->rho * c->rho * 1.01;
        rscale = bmax;
        K = c->filter_dd;
    }
    std::vector<double> allv;
    double worst = 0;
    for (int s = 0; s < nsec; ++s) {
        const int chi = which == 0 ? 0 : (s == 0 ? +1 : -1);
        cur = oprec;  // every sector starts in the work precision
        DF_TRY(prepare(oprec));
        if (which == 1 && c->chiral) {
            const double2 hc[3] = {make_double2(0, 0), make_double2(c->rho, 0), make_double2(chi * c->rho, 0)};
            DF_TRY(to_dev(c, hc, c->dscal + DSCAL_CHCO, sizeof hc, st));
            std::vector<double2> hb(3 * FB);
            for (int k = 0; k < 3; ++k)
                for (int q = 0; q < FB; ++q) hb[k * FB + q] = hc[k];
            DF_TRY(to_dev(c, hb.data(), c->dscal + DSCAL_CHCO + 16, hb.size() * sizeof(double2), st));
        }
        std::vector<double> v;
        double mr = 0;
        DF_TRY(chfsi(c, A, Awork, R, K, bmax, ns, nb, tol, rscale, which == 0, chi, 4242ull + 17 * which + s, W,
                     refine, v, sub(outv, s * ns, ns), &mr, st));
        allv.insert(allv.end(), v.begin(), v.end());
        worst = std::max(worst, mr);
    }
    std::vector<int> pick(allv.size());
    for (size_t i = 0; i < pick.size(); ++i) pick[i] = (int)i;
    std::stable_sort(pick.begin(), pick.end(), [&](int a, int b) { return std::fabs(allv[a]) < std::fabs(allv[b]); });
    pick.resize(nev);
    // the block and its rotation copy go before the eigenvectors' own storage is allocated (at 32^3 x 64
    // they are 150 GB), then the work fields that only the eigensolver uses
    cudaStreamSynchronize(st);
    field_free(c, &W.basis);
    field_free(c, &W.rot);
    DF_TRY(store_eigs(c, which, outv, pick, allv, st));
    cleanup();
    graphs_clear(c);  // captured applications may refer to the fields released here
    for (int slot : {(int)WS_LZ_WB, (int)WS_LZ_T, (int)WS_LZ_F0, (int)WS_LZ_F1, (int)WS_LZ_F2, (int)WS_LZ_F3})
        ws_release(c, slot);
    ws_release(c, WS_AUX1, P_F64, 16);
#undef DF_TRY
    (void)worst;
    return OV_OK;
}

// ---------------------------------------------------------------------------
// deflated CG with reliable updates
// ---------------------------------------------------------------------------
int net_apply_precond(ov_ctx* c, const FieldDesc& r, const FieldDesc& z, cudaStream_t st);
bool net_ready(const ov_ctx* c);
int net_record_pair(ov_ctx* c, const FieldDesc& r64, const FieldDesc& x64, cudaStream_t st);

int cg_impl(ov_ctx* c, const FieldDesc& b_in, const FieldDesc& x_out, double mass, double tol, int max_iter,
            int precond, int inner_prec, ov_solve_info* info, cudaStream_t st, bool warm)
{
    auto t0 = std::chrono::steady_clock::now();
    const int R = b_in.nrhs;
    const int Ps = inner_prec;
    // accurate arithmetic (true residuals, the accumulated solution): FP64 or double-float
    const int Ph = c->hi_prec;
    const bool sloppy = Ps != Ph;
    if (precond && !net_ready(c)) return set_err(c, OV_ESTATE, "cg: learned preconditioner requested but not trained");
    EigSet& X = c->eig[1];
    const int nd = X.nev;
    FieldDesc b = b_in, x = x_out;
    if (b_in.prec != Ph) {
        OV_TRY(ws_field(c, WS_CG_BH, Ph, R, &b));
        OV_TRY(ws_field(c, WS_CG_XH, Ph, R, &x));
        OV_TRY(convert(c, b_in, b, st));
        if (warm) OV_TRY(convert(c, x_out, x, st));
    }
    FieldDesc r, t, rs, ps, qs, xs, xt, zs, rold;
    OV_TRY(ws_field(c, WS_CG_R, Ph, R, &r));
    OV_TRY(ws_field(c, WS_CG_T, Ph, R, &t));
    OV_TRY(ws_field(c, WS_CG_U, Ph, R, &xt));
    if (sloppy) {
        OV_TRY(ws_field(c, WS_CG_RS, Ps, R, &rs));
    } else {
        rs = r;
    }
    OV_TRY(ws_field(c, WS_CG_XS, Ps, R, &xs));
    OV_TRY(ws_field(c, WS_CG_PS, Ps, R, &ps));
    OV_TRY(ws_field(c, WS_CG_QS, Ps, R, &qs));
    if (precond) {
        OV_TRY(ws_field(c, WS_CG_Z, Ps, R, &zs));
        OV_TRY(ws_field(c, WS_CG_P, Ps, R, &rold));
    }
    double2* dco = (double2*)(c->dscal + DSCAL_CGCO);  // per-rhs coefficients [K][R]
    double* dnr = c->dscal + DSCAL_NORM;              // per-rhs norms
    double2* ddt = (double2*)(c->dscal + DSCAL_DOT);   // per-rhs dots

    // deflation: mu_i(m) = (rho^2 - m^2/4) mu_i / rho^2 + m^2 (D^dag D = D + D^dag for the exact sign);
    // exact zero modes (mu_i <= 1e-10 mu_max) are left out of the solution (pseudo-inverse)
    std::vector<double> inv(nd, 0.0);
    {
        double mumax = 0;
        std::vector<double> mu(nd);
        for (int i = 0; i < nd; ++i) {
            mu[i] = (c->rho * c->rho - 0.25 * mass * mass) * X.vals[i] / (c->rho * c->rho) + mass * mass;
            mumax = std::max(mumax, mu[i]);
        }
        for (int i = 0; i < nd; ++i) inv[i] = mu[i] > 1e-10 * mumax ? 1.0 / mu[i] : 0.0;
    }
    if ((size_t)2 * nd * R * 2 > (size_t)DSCAL_COEF) return set_err(c, OV_EINVAL, "cg: nev * nrhs too large");
    FieldDesc xi64{}, xis{};
    if (nd) {
        OV_TRY(eig_vectors(c, 1, Ph, st, &xi64));
        OV_TRY(eig_vectors(c, 1, Ps, st, &xis));
    }
    auto project = [&](const FieldDesc& xiv, const FieldDesc& v) -> int {
        if (!nd) return OV_OK;
        OV_TRY(block_dots(c, xiv, nd, v, st));
        return block_sub(c, xiv, nd, v, st);
    };
    std::vector<double2> hb(R);
    OV_TRY(norm2(c, b, (double*)ddt, st));
    OV_TRY(to_host(c, ddt, hb.data(), R * sizeof(double2), st));
    std::vector<double> bn(R);
    for (int q = 0; q < R; ++q) bn[q] = hb[q].x > 0 ? std::sqrt(hb[q].x) : 1.0;

    // chiral-sector inner operator: every right-hand side must have definite chirality
    // (b^dag gamma5 b = +-|b|^2); the true residuals keep the full D^dag D
    const double2* dch = (const double2*)(c->dscal + DSCAL_CHCO);
    if (c->chiral) OV_TRY(chiral_setup(c, b, t, mass, st));
    // adaptive precision (Sec. V: adaptive CG): the inner operator may use a lower-degree polynomial; the
    // reliable updates recompute the true residual with the accurate one
    const int ipoly = c->adaptive_delta > 0 ? 1 : 0;
    // the one-sign form rests on sign^2 = 1; where the inner precision's rounding of a high-degree
    // polynomial breaks that by more than the smallest eigenvalue tolerates, the true residual stops
    // falling: then the solve continues with the two-sign operator (fallback bit 2)
    bool use_chiral = c->chiral != 0;
    int chiral_stalls = 0;
    auto inner_apply = [&](const FieldDesc& in, const FieldDesc& out) -> int {
        return use_chiral ? chiral_apply(c, in, out, mass, dch, st, ipoly) : normal_apply(c, in, out, mass, st, ipoly);
    };
    // In chiral mode every vector of the inner recursion must stay in its right-hand side's sector:
    // the one-sign operator acts on the other sector as m^2 (plus a coupling back), so rounding-level
    // components there would grow by ~rho^2/m^2 per cycle.  v <- (1 + chi gamma5) v / 2 after every
    // true residual and every preconditioner application (the network mixes chiralities).  Once the
    // solve has fallen back to the two-sign operator the projection stops: the true D^dag D couples
    // the sectors by as much as sign^2 differs from 1, and that part of the residual is what the
    // two-sign recursion has to remove.
    auto sector_project = [&](const FieldDesc& v) -> int {
        if (!use_chiral) return OV_OK;
        FieldDesc v2[2] = {v, v};
        return lincomb(c, v, 2, v2, nullptr, dch + 3 * R, 2, nullptr, st);
    };
    auto precond_apply = [&]() -> int {
        OV_TRY(net_apply_precond(c, rs, zs, st));
        return sector_project(zs);
    };

    std::vector<double> rr(R), rr_new(R), rmax(R), res(R, 1.0), rz(R);
    std::vector<char> done(R, 0);
    int iters = 0, updates = 0, fallback = 0;
    bool use_prec = precond != 0;

    // FP64 true residual r = b - A x, then the deflated restart (Eq. 9 on the current residual):
    // x += sum_i xi_i (xi_i^dag r) / mu_i and r <- r - sum_i xi_i (xi_i^dag r).  Repeating it at every
    // true residual removes the low-mode error even when the xi_i are approximate eigenvectors.
    // exact zero modes (excluded from the solution, the pseudo-inverse of reading 12): b's component along
    // them cannot be solved for, so the true residual is measured on their orthogonal complement
    int nzero = 0;
    for (int i = 0; i < nd; ++i) nzero += inv[i] == 0.0;
    // x <- x - sum_{zero modes} xi_i (xi_i^dag x): the pseudo-inverse has no component along them, and
    // the inner precision's rounding would otherwise leave one in the accumulated solution
    auto drop_zero_modes = [&](const FieldDesc& v) -> int {
        OV_TRY(block_dots(c, xi64, nd, v, st));
        std::vector<double2> h((size_t)nd * R);
        OV_TRY(to_host(c, c->dscal, h.data(), h.size() * sizeof(double2), st));
        for (int i = 0; i < nd; ++i)
            if (inv[i] != 0.0)
                for (int q = 0; q < R; ++q) h[(size_t)i * R + q] = make_double2(0, 0);
        OV_TRY(to_dev(c, h.data(), c->dscal, h.size() * sizeof(double2), st));
        FieldDesc none{};
        OV_CUDA(c, launch_proj_update(c->g, xi64, nd, (const double2*)c->dscal, nullptr, v, v, none, st));
        return OV_OK;
    };
    auto refresh = [&](bool& all_done) -> int {
        if (nzero) OV_TRY(drop_zero_modes(x));
        OV_TRY(normal_apply(c, x, t, mass, st));
        FieldDesc v2[2] = {b, t};
        double2 h2[2] = {make_double2(1, 0), make_double2(-1, 0)};
        OV_TRY(lincomb(c, r, 2, v2, h2, nullptr, 0, dnr, st));
        std::vector<double> nr(R);
        if (nzero) {
            OV_TRY(drop_zero_modes(r));
            std::vector<double2> hn(R);
            OV_TRY(norm2(c, r, (double*)ddt, st));
            OV_TRY(to_host(c, ddt, hn.data(), R * sizeof(double2), st));
            for (int q = 0; q < R; ++q) nr[q] = hn[q].x;
        } else {
            OV_TRY(to_host(c, dnr, nr.data(), R * sizeof(double), st));
        }
        all_done = true;
        for (int q = 0; q < R; ++q) {
            res[q] = std::sqrt(nr[q]) / bn[q];
            if (!std::isfinite(res[q])) return set_err(c, OV_ENAN, "cg: NaN/Inf in the true residual");
            if (res[q] <= tol) done[q] = 1;
            if (!done[q]) all_done = false;
        }
        ++updates;
        if (!all_done && nd) {
            OV_TRY(block_dots(c, xi64, nd, r, st));
            std::vector<double2> h((size_t)nd * R), hx((size_t)nd * R);
            OV_TRY(to_host(c, c->dscal, h.data(), h.size() * sizeof(double2), st));
            for (int i = 0; i < nd; ++i)
                for (int q = 0; q < R; ++q) {
                    double2& v = h[(size_t)i * R + q];
                    if (done[q]) v = make_double2(0, 0);
                    hx[(size_t)i * R + q] = make_double2(-v.x * inv[i], -v.y * inv[i]);
                }
            double2* cx = (double2*)c->dscal;
            double2* cr = cx + (size_t)nd * R;
            OV_TRY(to_dev(c, hx.data(), cx, hx.size() * sizeof(double2), st));
            OV_TRY(to_dev(c, h.data(), cr, h.size() * sizeof(double2), st));
            FieldDesc none{};
            OV_CUDA(c, launch_proj_update(c->g, xi64, nd, cx, nullptr, x, x, none, st));
            OV_CUDA(c, launch_proj_update(c->g, xi64, nd, cr, nullptr, r, r, none, st));
        }
        return net_record_pair(c, r, x, st);
    };
    auto sloppy_norms = [&](const FieldDesc& v, std::vector<double>& out) -> int {
        OV_TRY(norm2(c, v, (double*)ddt, st));
        std::vector<double2> h(R);
        OV_TRY(to_host(c, ddt, h.data(), R * sizeof(double2), st));
        for (int q = 0; q < R; ++q) out[q] = h[q].x;
        return OV_OK;
    };
    auto set_coef = [&](int K, const std::vector<double2>& h) -> int {
        return to_dev(c, h.data(), dco, (size_t)K * R * sizeof(double2), st);
    };
    // start (or restart) the search direction: p = z = M r (preconditioned) or p = r
    auto start_direction = [&]() -> int {
        if (use_prec) {
            OV_TRY(precond_apply());
            OV_TRY(project(xis, zs));
            OV_TRY(copy_field(c, zs, ps, st));
            OV_TRY(dot(c, rs, zs, ddt, st));
            std::vector<double2> h(R);
            OV_TRY(to_host(c, ddt, h.data(), R * sizeof(double2), st));
            for (int q = 0; q < R; ++q) rz[q] = h[q].x;
        } else {
            OV_TRY(copy_field(c, rs, ps, st));
            rz = rr;
        }
        return OV_OK;
    };

    if (!warm) OV_CUDA(c, cudaMemsetAsync(x.data, 0, x.rhs_bytes() * R, st));
    bool all_done = false;
    OV_TRY(refresh(all_done));
    const double delta = c->reliable_delta;  // reliable-update trigger: residual drop since the last update
    double prev_worst = 0;
    for (int q = 0; q < R; ++q) prev_worst = std::max(prev_worst, res[q]);
    if (!all_done) {
        if (sloppy) OV_TRY(convert(c, r, rs, st));
        OV_TRY(sector_project(rs));
        OV_CUDA(c, cudaMemsetAsync(xs.data, 0, xs.rhs_bytes() * R, st));
        if (xs.norm) OV_CUDA(c, cudaMemsetAsync(xs.norm, 0, (size_t)2 * xs.Vh * 4 * R, st));
        OV_TRY(sloppy_norms(rs, rr));
        for (int q = 0; q < R; ++q) rmax[q] = std::sqrt(rr[q]);
        OV_TRY(start_direction());
        int since = 0;
        std::vector<double2> co(2 * R);
        while (iters < max_iter) {
            OV_TRY(inner_apply(ps, qs));
            OV_TRY(dot(c, ps, qs, ddt, st));
            std::vector<double2> h(R);
            OV_TRY(to_host(c, ddt, h.data(), R * sizeof(double2), st));
            for (int q = 0; q < R; ++q) {
                const double a = (done[q] || !(h[q].x > 0)) ? 0.0 : rz[q] / h[q].x;
                co[q] = make_double2(1, 0);
                co[R + q] = make_double2(a, 0);
            }
            OV_TRY(set_coef(2, co));
            {
                FieldDesc v[2] = {xs, ps};
                OV_TRY(lincomb(c, xs, 2, v, nullptr, dco, 0, nullptr, st));
            }
            if (use_prec) OV_TRY(copy_field(c, rs, rold, st));
            for (int q = 0; q < R; ++q) co[R + q].x = -co[R + q].x;
            OV_TRY(set_coef(2, co));
            {
                FieldDesc v[2] = {rs, qs};
                OV_TRY(lincomb(c, rs, 2, v, nullptr, dco, 0, nullptr, st));
            }
            OV_TRY(project(xis, rs));
            OV_TRY(sloppy_norms(rs, rr_new));
            ++iters;
            ++since;
            bool trigger = since >= 200 || (use_prec && since >= 10);
            for (int q = 0; q < R; ++q) {
                if (done[q]) continue;
                if (!std::isfinite(rr_new[q])) return set_err(c, OV_ENAN, "cg: NaN/Inf in the residual");
                if (std::sqrt(rr_new[q]) <= tol * bn[q]) trigger = true;
                if (std::sqrt(rr_new[q]) < delta * rmax[q]) trigger = true;
            }
            bool restart = false;
            if (trigger) {
                // reliable update: x += xs (FP64), true residual, deflated restart
                OV_TRY(convert(c, xs, xt, st));
                FieldDesc v[2] = {x, xt};
                double2 h2[2] = {make_double2(1, 0), make_double2(1, 0)};
                OV_TRY(lincomb(c, x, 2, v, h2, nullptr, 0, nullptr, st));
                OV_CUDA(c, cudaMemsetAsync(xs.data, 0, xs.rhs_bytes() * R, st));
                if (xs.norm) OV_CUDA(c, cudaMemsetAsync(xs.norm, 0, (size_t)2 * xs.Vh * 4 * R, st));
                OV_TRY(refresh(all_done));
                if (verbose()) {
                    double w = 0;
                    for (int q = 0; q < R; ++q) w = std::max(w, res[q]);
                    fprintf(stderr, "[ov] cg iteration %d: true residual %.3e (update %d)\n", iters, w, updates);
                }
                if (all_done) break;
                double worst = 0;
                for (int q = 0; q < R; ++q)
                    if (!done[q]) worst = std::max(worst, res[q]);
                // learned-preconditioner stall rule: the true residual must drop by x0.9 per check
                if (use_prec && since >= 10 && worst > 0.9 * prev_worst) {
                    use_prec = false;
                    fallback |= 1;
                    restart = true;
                }
                // chiral-form stall rule: two reliable updates in a row that do not halve the true residual
                // (updates come when the inner residual has dropped by reliable_delta; with the learned
                // preconditioner they come every 10 iterations, and its own rule applies)
                if (use_chiral && !use_prec) {
                    chiral_stalls = worst > 0.5 * prev_worst ? chiral_stalls + 1 : 0;
                    if (chiral_stalls >= 2) {
                        use_chiral = false;
                        fallback |= 2;
                        restart = true;
                    }
                }
                prev_worst = worst;
                since = 0;
                if (sloppy) OV_TRY(convert(c, r, rs, st));
                OV_TRY(sector_project(rs));
                OV_TRY(sloppy_norms(rs, rr_new));
                for (int q = 0; q < R; ++q) rmax[q] = std::sqrt(rr_new[q]);
            }
            if (restart) {
                rr = rr_new;
                OV_TRY(start_direction());
                continue;
            }
            // next direction
            std::vector<double> rz_new(R);
            if (use_prec) {
                OV_TRY(precond_apply());
                OV_TRY(project(xis, zs));
                // flexible CG (Polak-Ribiere form): beta = z_new^dag (r_new - r_old) / (z_old^dag r_old)
                FieldDesc v[2] = {rs, rold};
                double2 h2[2] = {make_double2(1, 0), make_double2(-1, 0)};
                OV_TRY(lincomb(c, rold, 2, v, h2, nullptr, 0, nullptr, st));
                OV_TRY(dot(c, zs, rold, ddt, st));
                std::vector<double2> hh(R);
                OV_TRY(to_host(c, ddt, hh.data(), R * sizeof(double2), st));
                OV_TRY(dot(c, rs, zs, ddt, st));
                std::vector<double2> hz(R);
                OV_TRY(to_host(c, ddt, hz.data(), R * sizeof(double2), st));
                for (int q = 0; q < R; ++q) {
                    const double be = (trigger || rz[q] == 0) ? 0.0 : hh[q].x / rz[q];
                    co[q] = make_double2(1, 0);
                    co[R + q] = make_double2(be, 0);
                    rz_new[q] = hz[q].x;
                }
                OV_TRY(set_coef(2, co));
                FieldDesc w2[2] = {zs, ps};
                OV_TRY(lincomb(c, ps, 2, w2, nullptr, dco, 0, nullptr, st));
            } else {
                for (int q = 0; q < R; ++q) {
                    const double be = rr[q] > 0 ? rr_new[q] / rr[q] : 0.0;
                    co[q] = make_double2(1, 0);
                    co[R + q] = make_double2(be, 0);
                    rz_new[q] = rr_new[q];
                }
                OV_TRY(set_coef(2, co));
                FieldDesc w2[2] = {rs, ps};
                OV_TRY(lincomb(c, ps, 2, w2, nullptr, dco, 0, nullptr, st));
            }
            rr = rr_new;
            rz = rz_new;
        }
        if (!all_done && iters >= max_iter) {
            // fold the sloppy accumulation into x and report its true residual
            OV_TRY(convert(c, xs, xt, st));
            FieldDesc v[2] = {x, xt};
            double2 h2[2] = {make_double2(1, 0), make_double2(1, 0)};
            OV_TRY(lincomb(c, x, 2, v, h2, nullptr, 0, nullptr, st));
            OV_TRY(refresh(all_done));
        }
    }
    if (x.data != x_out.data) OV_TRY(convert(c, x, x_out, st));
    OV_CUDA(c, cudaStreamSynchronize(st));
    if (info) {
        memset(info, 0, sizeof *info);
        info->iterations = iters;
        info->reliable_updates = updates;
        info->fallback = fallback;
        info->nrhs = R;
        for (int q = 0; q < R && q < 64; ++q) info->true_residual[q] = res[q];
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    bool ok = true;
    for (int q = 0; q < R; ++q) ok = ok && res[q] <= tol;
    if (!ok) return set_err(c, OV_ENOTCONV, "cg: not converged after %d iterations", iters);
    return OV_OK;
}

// ---------------------------------------------------------------------------
// multi-mass solve (Sec. II: one multi-shifted CG for the propagators of several masses)
// ---------------------------------------------------------------------------
// With sign^2 = 1, D(m)^dag D(m) = a_m (D(0)^dag D(0) + s_m), a_m = 1 - m^2 / (4 rho^2), s_m = m^2 / a_m
// (Eq. 8 and D^dag D = rho (D + D^dag)), so every mass shares the Krylov space of D(0)^dag D(0).  Step 1:
// on the complement of the stored D^dag D modes xi_i, the shifted systems (A0 + s_k) y_k = b_h are solved by
// one CG recursion on A0 in the inner precision, whose shifted residuals are collinear with the base
// residual, r_k = z_k r (shifted-system CG, Jegerlehner 1996); each (mass, right-hand side) stops once
// |z_k| |r| <= tol_in |b_h|.  Step 2: x_k = y_k / a_k + sum_i xi_i (xi_i^dag b) / (a_k mu_i + m_k^2) (Eq. 9)
// in the accurate precision.  Step 3: the identity above holds only up to the polynomial's error, so each
// mass is refined by the deflated mixed-precision CG with reliable updates (cg_impl, warm start), whose
// true residuals use the full two-sign D(m_k)^dag D(m_k).  Output 1 turns x_k into D(m_k)^-1 b =
// D(m_k)^dag x_k = gamma5 D(m_k) gamma5 x_k, output 2 into the propagator (1 - D/2) D(m_k)^-1 b with
// D = D(0)/rho, computed as z - D(0) z / (2 rho).
int multimass_impl(ov_ctx* c, const FieldDesc& b_in, const FieldDesc* xout, int nmass, const double* masses,
                   double tol, int max_iter, int inner_prec, int output, ov_solve_info* info, cudaStream_t st)
{
    auto t0 = std::chrono::steady_clock::now();
    const int R = b_in.nrhs, M = nmass, Ps = inner_prec, Ph = c->hi_prec;
    const double rho = c->rho;
    EigSet& X = c->eig[1];
    const int nd = X.nev;
    if ((size_t)(2 * M + 2) * R * 2 > (size_t)(DSCAL_NORM - DSCAL_CGCO) || (size_t)2 * nd * R * 2 > DSCAL_COEF)
        return set_err(c, OV_EINVAL, "multimass: too many masses, right-hand sides or modes");
    std::vector<double> am(M), sm(M);
    for (int k = 0; k < M; ++k) {
        am[k] = 1.0 - masses[k] * masses[k] / (4.0 * rho * rho);
        if (!(am[k] > 0)) return set_err(c, OV_EINVAL, "multimass: mass %g >= 2 rho", masses[k]);
        sm[k] = masses[k] * masses[k] / am[k];
    }
    // work fields: accurate b, inner r, p, q, and per mass p_k, y_k
    FieldDesc b = b_in, r, p, q;
    if (b_in.prec != Ph) {
        OV_TRY(ws_field(c, WS_CG_BH, Ph, R, &b));
        OV_TRY(convert(c, b_in, b, st));
    }
    OV_TRY(ws_field(c, WS_CG_RS, Ps, R, &r));
    OV_TRY(ws_field(c, WS_CG_PS, Ps, R, &p));
    OV_TRY(ws_field(c, WS_CG_QS, Ps, R, &q));
    std::vector<FieldDesc> pk(M), yk(M);
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (auto& f : pk) field_free(c, &f);
        for (auto& f : yk) field_free(c, &f);
    };
#define MM_TRY(x)              \
    do {                       \
        int s__ = (x);         \
        if (s__ != OV_OK) {    \
            release();         \
            return s__;        \
        }                      \
    } while (0)
    for (int k = 0; k < M; ++k) {
        MM_TRY(field_alloc(c, Ps, R, &pk[k]));
        MM_TRY(field_alloc(c, Ps, R, &yk[k]));
    }
    FieldDesc xi64{}, xis{};
    if (nd) {
        MM_TRY(eig_vectors(c, 1, Ph, st, &xi64));
        MM_TRY(eig_vectors(c, 1, Ps, st, &xis));
    }
    double2* dco = (double2*)(c->dscal + DSCAL_CGCO);
    double2* ddt = (double2*)(c->dscal + DSCAL_DOT);
    double* dnr = c->dscal + DSCAL_NORM;
    // low-mode coefficients pb[i][q] = xi_i^dag b_q, and b_h = b - sum_i xi_i pb_i
    std::vector<double2> pb((size_t)nd * R);
    FieldDesc bh;
    MM_TRY(ws_field(c, WS_CG_T, Ph, R, &bh));
    MM_TRY(copy_field(c, b, bh, st));
    if (nd) {
        MM_TRY(block_dots(c, xi64, nd, b, st));
        MM_TRY(to_host(c, c->dscal, pb.data(), pb.size() * sizeof(double2), st));
        MM_TRY(block_sub(c, xi64, nd, bh, st));
    }
    // chiral mode: the inner operator A0 is the one-sign form on each source's sector
    if (c->chiral) {
        FieldDesc tmp;
        MM_TRY(ws_field(c, WS_CG_U, Ph, R, &tmp));  // a field of bh's precision for the chirality test
        MM_TRY(chiral_setup(c, bh, tmp, 0.0, st));
    }
    const double2* dch = (const double2*)(c->dscal + DSCAL_CHCO);
    const int ipoly = c->adaptive_delta > 0 ? 1 : 0;
    auto A0 = [&](const FieldDesc& in, const FieldDesc& out) -> int {
        return c->chiral ? chiral_apply(c, in, out, 0.0, dch, st, ipoly) : normal_apply(c, in, out, 0.0, st, ipoly);
    };
    MM_TRY(convert(c, bh, r, st));
    MM_TRY(copy_field(c, r, p, st));
    for (int k = 0; k < M; ++k) {
        MM_TRY(copy_field(c, r, pk[k], st));
        MM_TRY(cudaMemsetAsync(yk[k].data, 0, yk[k].rhs_bytes() * R, st) == cudaSuccess ? OV_OK : OV_ECUDA);
        if (yk[k].norm) MM_TRY(cudaMemsetAsync(yk[k].norm, 0, (size_t)2 * yk[k].Vh * 4 * R, st) == cudaSuccess ? OV_OK : OV_ECUDA);
    }
    std::vector<double> rr(R), bhn(R);
    {
        std::vector<double2> h(R);
        MM_TRY(norm2(c, r, (double*)ddt, st));
        MM_TRY(to_host(c, ddt, h.data(), R * sizeof(double2), st));
        for (int j = 0; j < R; ++j) rr[j] = bhn[j] = h[j].x;
        for (int j = 0; j < R; ++j) bhn[j] = std::sqrt(bhn[j]);
    }
    // the inner precision cannot resolve residuals below its rounding: the shifted solve stops there and
    // the refinement (FP64 or double-float true residuals) finishes the job
    const double tol_in = std::max(tol, wide(Ps) ? tol : (Ps == P_F32 ? 1e-6 : 1e-3));
    // shifted-CG scalars per (mass, rhs): z, z_old, and the base recursion's alpha_old, beta_old per rhs
    std::vector<double> z((size_t)M * R, 1.0), zo((size_t)M * R, 1.0), zn((size_t)M * R, 1.0);
    std::vector<double> aold(R, 1.0), bold(R, 0.0);
    std::vector<char> active((size_t)M * R, 1);
    for (int j = 0; j < R; ++j)
        if (!(bhn[j] > 0))
            for (int k = 0; k < M; ++k) active[(size_t)k * R + j] = 0;  // b in span(xi): the low modes solve it
    int iters = 0;
    std::vector<double2> co((size_t)(2 * M + 2) * R);
    while (iters < max_iter) {
        bool any = false;
        for (char a : active) any = any || a;
        if (!any) break;
        MM_TRY(A0(p, q));
        if (nd) {  // q <- (1 - sum xi xi^dag) q: the recursion stays on the deflated complement
            MM_TRY(block_dots(c, xis, nd, q, st));
            MM_TRY(block_sub(c, xis, nd, q, st));
        }
        std::vector<double2> h(R);
        MM_TRY(dot(c, p, q, ddt, st));
        MM_TRY(to_host(c, ddt, h.data(), R * sizeof(double2), st));
        std::vector<double> alpha(R, 0.0);
        for (int j = 0; j < R; ++j) {
            bool live = false;
            for (int k = 0; k < M; ++k) live = live || active[(size_t)k * R + j];
            alpha[j] = (live && h[j].x > 0) ? rr[j] / h[j].x : 0.0;
            if (!std::isfinite(alpha[j])) {
                release();
                return set_err(c, OV_ENAN, "multimass: NaN/Inf in the recursion");
            }
        }
        // y_k += alpha_k p_k, alpha_k = alpha z_k' / z_k (coefficient blocks [k][2][R])
        for (int k = 0; k < M; ++k)
            for (int j = 0; j < R; ++j) {
                const size_t kj = (size_t)k * R + j;
                zn[kj] = z[kj];
                double ak = 0.0;
                if (active[kj] && alpha[j] != 0.0) {
                    zn[kj] = z[kj] * zo[kj] * aold[j] /
                             (alpha[j] * bold[j] * (zo[kj] - z[kj]) + zo[kj] * aold[j] * (1.0 + sm[k] * alpha[j]));
                    ak = alpha[j] * zn[kj] / z[kj];
                }
                co[(size_t)(2 * k) * R + j] = make_double2(1, 0);
                co[(size_t)(2 * k + 1) * R + j] = make_double2(ak, 0);
            }
        // r -= alpha q (with |r|^2)
        for (int j = 0; j < R; ++j) {
            co[(size_t)(2 * M) * R + j] = make_double2(1, 0);
            co[(size_t)(2 * M + 1) * R + j] = make_double2(-alpha[j], 0);
        }
        MM_TRY(to_dev(c, co.data(), dco, co.size() * sizeof(double2), st));
        for (int k = 0; k < M; ++k) {
            FieldDesc v[2] = {yk[k], pk[k]};
            MM_TRY(lincomb(c, yk[k], 2, v, nullptr, dco + (size_t)(2 * k) * R, 0, nullptr, st));
        }
        {
            FieldDesc v[2] = {r, q};
            MM_TRY(lincomb(c, r, 2, v, nullptr, dco + (size_t)(2 * M) * R, 0, dnr, st));
        }
        std::vector<double> rn(R);
        MM_TRY(to_host(c, dnr, rn.data(), R * sizeof(double), st));  // also orders the coefficient reuse below
        ++iters;
        std::vector<double> beta(R, 0.0);
        for (int j = 0; j < R; ++j) {
            if (!std::isfinite(rn[j])) {
                release();
                return set_err(c, OV_ENAN, "multimass: NaN/Inf in the residual");
            }
            beta[j] = (alpha[j] != 0.0 && rr[j] > 0) ? rn[j] / rr[j] : 0.0;
        }
        // p_k = z_k' r + beta_k p_k, beta_k = beta (z_k' / z_k)^2; a finished (mass, rhs) keeps p_k, y_k
        for (int k = 0; k < M; ++k)
            for (int j = 0; j < R; ++j) {
                const size_t kj = (size_t)k * R + j;
                double zr = 0.0, bk = 1.0;
                if (active[kj] && alpha[j] != 0.0) {
                    zr = zn[kj];
                    bk = beta[j] * (zn[kj] / z[kj]) * (zn[kj] / z[kj]);
                    if (std::fabs(zn[kj]) * std::sqrt(rn[j]) <= tol_in * bhn[j]) active[kj] = 0;
                }
                co[(size_t)(2 * k) * R + j] = make_double2(zr, 0);
                co[(size_t)(2 * k + 1) * R + j] = make_double2(bk, 0);
                if (zn[kj] != z[kj]) {
                    zo[kj] = z[kj];
                    z[kj] = zn[kj];
                }
            }
        for (int j = 0; j < R; ++j) {
            co[(size_t)(2 * M) * R + j] = make_double2(1, 0);
            co[(size_t)(2 * M + 1) * R + j] = make_double2(alpha[j] != 0.0 ? beta[j] : 1.0, 0);
            if (alpha[j] != 0.0) {
                aold[j] = alpha[j];
                bold[j] = beta[j];
                rr[j] = rn[j];
            }
        }
        MM_TRY(to_dev(c, co.data(), dco, co.size() * sizeof(double2), st));
        for (int k = 0; k < M; ++k) {
            FieldDesc v[2] = {r, pk[k]};
            MM_TRY(lincomb(c, pk[k], 2, v, nullptr, dco + (size_t)(2 * k) * R, 0, nullptr, st));
        }
        {
            FieldDesc v[2] = {r, p};
            MM_TRY(lincomb(c, p, 2, v, nullptr, dco + (size_t)(2 * M) * R, 0, nullptr, st));
        }
        if (c->chiral) {  // keep the recursion on each source's sector (rounding leaks out of it)
            FieldDesc v2[2] = {p, p};
            MM_TRY(lincomb(c, p, 2, v2, nullptr, dch + 3 * R, 2, nullptr, st));
        }
        if (verbose() && iters % 50 == 0) {
            double w = 0;
            for (int j = 0; j < R; ++j) w = std::max(w, std::sqrt(rn[j]) / bhn[j]);
            fprintf(stderr, "[ov] multimass iteration %d: base residual %.3e\n", iters, w);
        }
    }
    // x_k = y_k / a_k + sum_i xi_i pb_i / (a_k mu_i + m_k^2) in the accurate precision
    FieldDesc xt;
    MM_TRY(ws_field(c, WS_CG_U, Ph, R, &xt));
    for (int k = 0; k < M; ++k) {
        MM_TRY(convert(c, yk[k], xt, st));
        const double2 hs = make_double2(1.0 / am[k], 0);
        MM_TRY(lincomb(c, xout[k], 1, &xt, &hs, nullptr, 0, nullptr, st));
        if (nd) {
            std::vector<double2> cx((size_t)nd * R);
            for (int i = 0; i < nd; ++i) {
                const double muk = am[k] * X.vals[i] + masses[k] * masses[k];
                const double inv = muk > 1e-10 * (am[k] * X.vals[nd - 1] + masses[k] * masses[k]) ? 1.0 / muk : 0.0;
                for (int j = 0; j < R; ++j) {
                    const double2 v = pb[(size_t)i * R + j];
                    cx[(size_t)i * R + j] = make_double2(-v.x * inv, -v.y * inv);  // proj_update subtracts
                }
            }
            MM_TRY(to_dev(c, cx.data(), c->dscal, cx.size() * sizeof(double2), st));
            FieldDesc none{};
            MM_TRY(launch_proj_update(c->g, xi64, nd, (const double2*)c->dscal, nullptr, xout[k], xout[k], none, st) ==
                           cudaSuccess
                       ? OV_OK
                       : OV_ECUDA);
            MM_TRY(cudaStreamSynchronize(st) == cudaSuccess ? OV_OK : OV_ECUDA);
        }
    }
    release();
#undef MM_TRY
    // refinement per mass (warm start), then the requested output
    int worst = OV_OK;
    for (int k = 0; k < M; ++k) {
        ov_solve_info inf{};
        const int left = std::max(1, max_iter - iters);
        int sk = cg_impl(c, b_in, xout[k], masses[k], tol, left, 0, Ps, &inf, st, true);
        if (sk != OV_OK && sk != OV_ENOTCONV) return sk;
        if (sk != OV_OK) worst = sk;
        if (info) {
            info[k] = inf;
            info[k].iterations += iters;
        }
        if (output >= 1) {
            // z = D(m)^dag x = gamma5 D(m) gamma5 x
            FieldDesc t1, t2;
            OV_TRY(ws_field(c, WS_AUX1, xout[k].prec, R, &t1));
            OV_TRY(ws_field(c, WS_CG_U, xout[k].prec, R, &t2));
            const double2 one = make_double2(1, 0);
            OV_TRY(lincomb(c, t1, 1, &xout[k], &one, nullptr, 1, nullptr, st));  // t1 = gamma5 x
            if (output == 1) {
                OV_TRY(overlap_g5_apply(c, t1, xout[k], masses[k], 1, st));
            } else {
                OV_TRY(overlap_g5_apply(c, t1, t2, masses[k], 1, st));   // t2 = z
                OV_TRY(overlap_apply(c, t2, t1, 0.0, st));                      // t1 = D(0) z
                FieldDesc v[2] = {t2, t1};
                const double2 h[2] = {make_double2(1, 0), make_double2(-0.5 / rho, 0)};
                OV_TRY(lincomb(c, xout[k], 2, v, h, nullptr, 0, nullptr, st));
            }
        }
    }
    OV_CUDA(c, cudaStreamSynchronize(st));
    if (info) {
        const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int k = 0; k < M; ++k) info[k].seconds = sec;
    }
    return worst == OV_OK ? OV_OK : set_err(c, worst, "multimass: a mass did not converge");
}

// ---------------------------------------------------------------------------
// rational sign (Eq. 12): s = sum_i b_i (Q^2 + c_i)^-1 src by multi-shift CG
// ---------------------------------------------------------------------------
// One CG on the base system (Q^2 + c_0) x = src, c_0 the smallest pole; the others are shifted systems
// (Q^2 + c_0 + sigma_i) x_i = src, sigma_i = c_i - c_0 >= 0, whose residuals stay collinear with the base
// residual, r_i = z_i r (Jegerlehner 1996; the same recurrences as the multi-mass solve).  Single pass
// (the paper's "single pass"): the 2n shifted vectors p_i, x_i are updated every iteration and summed at
// the end.  Double pass (Neuberger): the first pass runs the base CG alone and records its scalars; the
// shifted scalars follow on the host, and with them the coefficient g_j of every base residual r_j in
// s = sum_i b_i x_i (x_i = sum_k a_i^k p_i^k, p_i^k = zeta_i^k r_k + beta_i^(k-1) p_i^(k-1), so the
// coefficient of r_j in x_i is zeta_i^j G_i^j with G_i^j = a_i^j + beta_i^j G_i^(j+1)); the second pass
// repeats the base recursion with the recorded scalars (bit for bit the same r_j) and accumulates
// s = sum_j g_j r_j: twice the dslash applications, three vector updates per iteration instead of 2n + 2.
// Q^2 = H_w^2 / lambda_max^2; each application is two dslash launches, the shift fused into the second.
int rational_solve(ov_ctx* c, const FieldDesc& src, const FieldDesc& s, int gprec, cudaStream_t st)
{
    const int R = src.nrhs, P = src.prec, n = (int)c->rb.size();
    const double lam2 = c->lmax * c->lmax, aw = 4.0 - c->rho;
    int i0 = 0;
    for (int i = 1; i < n; ++i)
        if (c->rc[i] < c->rc[i0]) i0 = i;
    const double c0 = c->rc[i0];
    std::vector<double> sg(n);
    for (int i = 0; i < n; ++i) sg[i] = c->rc[i] - c0;
    const double tol = P == P_F64 || P == P_DF64 ? c->rational_tol : std::max(c->rational_tol, 1e-6);
    FieldDesc r, p, q, t;
    OV_TRY(ws_field(c, WS_RR, P, R, &r));
    OV_TRY(ws_field(c, WS_RP, P, R, &p));
    OV_TRY(ws_field(c, WS_RQ, P, R, &q));
    OV_TRY(ws_field(c, WS_RT, P, R, &t));
    auto Aop = [&](const FieldDesc& in, const FieldDesc& out) -> int {  // (Q^2 + c_0) in
        OV_TRY(dslash_apply(c, in, t, aw, -0.5, 1, 0, 0, nullptr, nullptr, st, gprec));
        FieldDesc y[1] = {in};
        double sy[1] = {c0};
        return dslash_apply(c, t, out, aw / lam2, -0.5 / lam2, 1, 0, 1, y, sy, st, gprec);
    };
    const bool single = c->rational_pass == 1;
    std::vector<FieldDesc> xs, ps;
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (auto& f : xs) field_free(c, &f);
        for (auto& f : ps) field_free(c, &f);
    };
#define RS_TRY(x)             \
    do {                      \
        int s__ = (x);        \
        if (s__ != OV_OK) {   \
            release();        \
            return s__;       \
        }                     \
    } while (0)
    if (single) {
        xs.resize(n);
        ps.resize(n);
        for (int i = 0; i < n; ++i) {
            RS_TRY(field_alloc(c, P, R, &xs[i]));
            RS_TRY(field_alloc(c, P, R, &ps[i]));
            RS_TRY(copy_field(c, src, ps[i], st));
            RS_TRY(cudaMemsetAsync(xs[i].data, 0, xs[i].rhs_bytes() * R, st) == cudaSuccess ? OV_OK : OV_ECUDA);
            if (xs[i].norm)
                RS_TRY(cudaMemsetAsync(xs[i].norm, 0, (size_t)2 * xs[i].Vh * 4 * R, st) == cudaSuccess ? OV_OK
                                                                                                       : OV_ECUDA);
        }
    }
    // device coefficient blocks ([K][R] double2 per lincomb), grown as needed
    auto coef_buf = [&](size_t n2) -> double2* {
        const size_t bytes = n2 * sizeof(double2);
        if (bytes > c->rcoef_bytes) {
            cudaStreamSynchronize(st);
            if (c->rcoef) dev_free(c, c->rcoef, c->rcoef_bytes);
            c->rcoef = nullptr;
            c->rcoef_bytes = 0;
            void* pp = nullptr;
            if (dev_alloc(c, &pp, bytes) != OV_OK) return nullptr;
            c->rcoef = pp;
            c->rcoef_bytes = bytes;
        }
        return (double2*)c->rcoef;
    };
    double2* ddt = (double2*)(c->dscal + DSCAL_DOT);
    double* dnr = c->dscal + DSCAL_NORM;
    RS_TRY(copy_field(c, src, r, st));
    RS_TRY(copy_field(c, src, p, st));
    std::vector<double> rr(R), bn(R);
    {
        std::vector<double2> h(R);
        RS_TRY(norm2(c, r, (double*)ddt, st));
        RS_TRY(to_host(c, ddt, h.data(), R * sizeof(double2), st));
        for (int j = 0; j < R; ++j) {
            rr[j] = h[j].x;
            bn[j] = std::sqrt(h[j].x);
        }
    }
    // per (shift, rhs) scalars; the recorded base scalars and shifted coefficients for the second pass
    std::vector<double> z((size_t)n * R, 1.0), zo((size_t)n * R, 1.0), zn((size_t)n * R, 1.0);
    std::vector<double> aold(R, 1.0), bold(R, 0.0);
    std::vector<char> act((size_t)n * R, 1), live(R, 1);
    for (int j = 0; j < R; ++j)
        if (!(bn[j] > 0)) live[j] = 0;
    std::vector<std::vector<double>> A_k, B_k;                     // base alpha, beta per iteration [R]
    std::vector<std::vector<double>> ZE, AI, BI;                    // zeta_i^k, a_i^k, beta_i^k [n*R]
    ZE.push_back(std::vector<double>((size_t)n * R, 1.0));          // zeta^0 = 1
    int it = 0;
    const int itmax = 20000;
    for (; it < itmax; ++it) {
        bool any = false;
        for (int j = 0; j < R; ++j) any = any || live[j];
        if (!any) break;
        RS_TRY(Aop(p, q));
        std::vector<double2> h(R);
        RS_TRY(dot(c, p, q, ddt, st));
        RS_TRY(to_host(c, ddt, h.data(), R * sizeof(double2), st));
        std::vector<double> alpha(R, 0.0);
        for (int j = 0; j < R; ++j) {
            alpha[j] = (live[j] && h[j].x > 0) ? rr[j] / h[j].x : 0.0;
            if (!std::isfinite(alpha[j])) {
                release();
                return set_err(c, OV_ENAN, "rational sign: NaN/Inf in the recursion");
            }
        }
        std::vector<double> ai((size_t)n * R, 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < R; ++j) {
                const size_t ij = (size_t)i * R + j;
                zn[ij] = z[ij];
                if (act[ij] && alpha[j] != 0.0) {
                    zn[ij] = z[ij] * zo[ij] * aold[j] /
                             (alpha[j] * bold[j] * (zo[ij] - z[ij]) + zo[ij] * aold[j] * (1.0 + sg[i] * alpha[j]));
                    ai[ij] = alpha[j] * zn[ij] / z[ij];
                }
            }
        if (single) {  // x_i += a_i p_i
            double2* dc = coef_buf((size_t)2 * n * R);
            if (!dc) {
                release();
                return OV_ENOMEM;
            }
            std::vector<double2> hc((size_t)2 * n * R);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < R; ++j) {
                    hc[(size_t)(2 * i) * R + j] = make_double2(1, 0);
                    hc[(size_t)(2 * i + 1) * R + j] = make_double2(ai[(size_t)i * R + j], 0);
                }
            RS_TRY(to_dev(c, hc.data(), dc, hc.size() * sizeof(double2), st));
            for (int i = 0; i < n; ++i) {
                FieldDesc v[2] = {xs[i], ps[i]};
                RS_TRY(lincomb(c, xs[i], 2, v, nullptr, dc + (size_t)(2 * i) * R, 0, nullptr, st));
            }
        }
        // r -= alpha q, with |r|^2
        std::vector<double2> hb(2 * R);
        for (int j = 0; j < R; ++j) {
            hb[j] = make_double2(1, 0);
            hb[R + j] = make_double2(-alpha[j], 0);
        }
        double2* dco = (double2*)(c->dscal + DSCAL_CGCO);
        RS_TRY(to_dev(c, hb.data(), dco, hb.size() * sizeof(double2), st));
        {
            FieldDesc v[2] = {r, q};
            RS_TRY(lincomb(c, r, 2, v, nullptr, dco, 0, dnr, st));
        }
        std::vector<double> rn(R);
        RS_TRY(to_host(c, dnr, rn.data(), R * sizeof(double), st));
        std::vector<double> beta(R, 1.0), bi((size_t)n * R, 1.0);
        for (int j = 0; j < R; ++j) {
            if (!std::isfinite(rn[j])) {
                release();
                return set_err(c, OV_ENAN, "rational sign: NaN/Inf in the residual");
            }
            if (alpha[j] != 0.0) beta[j] = rr[j] > 0 ? rn[j] / rr[j] : 0.0;
        }
        std::vector<double> zeta_next((size_t)n * R, 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < R; ++j) {
                const size_t ij = (size_t)i * R + j;
                if (act[ij] && alpha[j] != 0.0) {
                    bi[ij] = beta[j] * (zn[ij] / z[ij]) * (zn[ij] / z[ij]);
                    zeta_next[ij] = zn[ij];
                    if (std::fabs(zn[ij]) * std::sqrt(rn[j]) <= tol * bn[j]) act[ij] = 0;
                } else {
                    bi[ij] = 1.0;  // p_i is frozen (its x_i no longer moves)
                }
                if (zn[ij] != z[ij]) {
                    zo[ij] = z[ij];
                    z[ij] = zn[ij];
                }
            }
        if (single) {  // p_i = zn r + beta_i p_i
            double2* dc = coef_buf((size_t)2 * n * R);
            std::vector<double2> hc((size_t)2 * n * R);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < R; ++j) {
                    const size_t ij = (size_t)i * R + j;
                    const bool mv = bi[ij] != 1.0 || zeta_next[ij] != 0.0;
                    hc[(size_t)(2 * i) * R + j] = make_double2(mv ? zeta_next[ij] : 0.0, 0);
                    hc[(size_t)(2 * i + 1) * R + j] = make_double2(bi[ij], 0);
                }
            RS_TRY(to_dev(c, hc.data(), dc, hc.size() * sizeof(double2), st));
            for (int i = 0; i < n; ++i) {
                FieldDesc v[2] = {r, ps[i]};
                RS_TRY(lincomb(c, ps[i], 2, v, nullptr, dc + (size_t)(2 * i) * R, 0, nullptr, st));
            }
        }
        // p = r + beta p
        for (int j = 0; j < R; ++j) {
            hb[j] = make_double2(1, 0);
            hb[R + j] = make_double2(alpha[j] != 0.0 ? beta[j] : 1.0, 0);
            if (alpha[j] != 0.0) {
                aold[j] = alpha[j];
                bold[j] = beta[j];
                rr[j] = rn[j];
            }
            bool done = true;
            for (int i = 0; i < n; ++i) done = done && !act[(size_t)i * R + j];
            if (done) live[j] = 0;
        }
        RS_TRY(to_dev(c, hb.data(), dco, hb.size() * sizeof(double2), st));
        {
            FieldDesc v[2] = {r, p};
            RS_TRY(lincomb(c, p, 2, v, nullptr, dco, 0, nullptr, st));
        }
        A_k.push_back(alpha);
        B_k.push_back(beta);
        AI.push_back(ai);
        BI.push_back(bi);
        ZE.push_back(zeta_next);
    }
    c->rational_iters = it;
    if (it >= itmax) {
        release();
        return set_err(c, OV_ENOTCONV, "rational sign: multi-shift CG not converged in %d iterations", itmax);
    }
    if (single) {  // s = sum_i b_i x_i, four fields per launch (s itself after the first)
        int i = 0;
        bool first = true;
        while (i < n) {
            FieldDesc v[4];
            double2 hc[4];
            int K = 0;
            if (!first) {
                v[K] = s;
                hc[K++] = make_double2(1, 0);
            }
            while (K < 4 && i < n) {
                v[K] = xs[i];
                hc[K++] = make_double2(c->rb[i], 0);
                ++i;
            }
            RS_TRY(lincomb(c, s, K, v, hc, nullptr, 0, nullptr, st));
            first = false;
        }
        release();
        return OV_OK;
    }
    // double pass: g_j per rhs from the recorded scalars, then the repeated base recursion
    const int Kit = it;
    std::vector<double> g((size_t)(Kit + 1) * R, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < R; ++j) {
            double G = 0.0;  // G_i^(K) = 0
            for (int k = Kit - 1; k >= 0; --k) {
                const size_t ij = (size_t)i * R + j;
                G = AI[k][ij] + BI[k][ij] * G;
                g[(size_t)k * R + j] += c->rb[i] * ZE[k][ij] * G;
            }
        }
    double2* dc = coef_buf((size_t)6 * R * (Kit + 1));
    if (!dc) {
        release();
        return OV_ENOMEM;
    }
    std::vector<double2> hc((size_t)6 * R * (Kit + 1));
    for (int k = 0; k <= Kit; ++k)
        for (int j = 0; j < R; ++j) {
            const double al = k < Kit ? A_k[k][j] : 0.0, be = k < Kit ? B_k[k][j] : 1.0;
            double2* blk = hc.data() + (size_t)6 * R * k;
            blk[j] = make_double2(1, 0);                  // r_{k+1} = r_k - alpha_k q
            blk[R + j] = make_double2(-al, 0);
            blk[2 * R + j] = make_double2(1, 0);          // p_{k+1} = r_{k+1} + beta_k p_k
            blk[3 * R + j] = make_double2(be, 0);
            blk[4 * R + j] = make_double2(1, 0);          // s += g_{k+1} r_{k+1}
            blk[5 * R + j] = make_double2(k + 1 <= Kit ? g[(size_t)std::min(k + 1, Kit) * R + j] : 0.0, 0);
        }
    RS_TRY(to_dev(c, hc.data(), dc, hc.size() * sizeof(double2), st));
    RS_TRY(copy_field(c, src, r, st));
    RS_TRY(copy_field(c, src, p, st));
    {
        std::vector<double2> g0(R);
        for (int j = 0; j < R; ++j) g0[j] = make_double2(g[j], 0);
        double2* dco = (double2*)(c->dscal + DSCAL_CGCO);
        RS_TRY(to_dev(c, g0.data(), dco, R * sizeof(double2), st));
        FieldDesc v[1] = {src};
        RS_TRY(lincomb(c, s, 1, v, nullptr, dco, 0, nullptr, st));  // s = g_0 r_0
    }
    for (int k = 0; k < Kit; ++k) {
        const double2* blk = dc + (size_t)6 * R * k;
        RS_TRY(Aop(p, q));
        FieldDesc v1[2] = {r, q};
        RS_TRY(lincomb(c, r, 2, v1, nullptr, blk, 0, nullptr, st));
        FieldDesc v2[2] = {r, p};
        RS_TRY(lincomb(c, p, 2, v2, nullptr, blk + 2 * R, 0, nullptr, st));
        FieldDesc v3[2] = {s, r};
        RS_TRY(lincomb(c, s, 2, v3, nullptr, blk + 4 * R, 0, nullptr, st));
    }
    release();
#undef RS_TRY
    return OV_OK;
}

}  // namespace ov
