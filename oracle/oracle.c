/*
 * FP64 CPU oracle for the overlap-operator hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so the tests, the smoke check and the CPU-baseline
 * leg of the benchmark can check the CUDA library against a plain, slow,
 * obviously correct restatement of the method.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Everything is double precision, canonical (non even/odd) layout:
 *   gauge  U   : complex [Lt][Lz][Ly][Lx][mu=0..3 (x,y,z,t)][3][3]
 *   spinor psi : complex [Lt][Lz][Ly][Lx][spin 4][colour 3]
 * dims[] = {Lx, Ly, Lz, Lt}; bc[mu] is a real phase (+1 periodic, -1
 * antiperiodic) multiplying every hop that crosses the boundary in mu.
 *
 * Gamma matrices: Euclidean chiral basis, gamma_k = [[0,-i s_k],[i s_k,0]]
 * (k=1,2,3), gamma_4 = [[0,1],[1,0]], gamma_5 = g1 g2 g3 g4 = diag(1,1,-1,-1).
 * The paper fixes only "chiral" (Sec. V); the explicit matrices are this
 * project's reading.
 *
 * Parity status of each function (what pins it) is listed in the Python
 * wrapper oracle/__init__.py.
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* OpenMP threads the parallel loops use, and a way to set them (CPU timing) */
int or_threads(void) { return omp_get_max_threads(); }
void or_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }

/* ------------------------------------------------------------------ */
/* gamma matrices                                                       */
/* ------------------------------------------------------------------ */
static cplx G[5][4][4]; /* G[0..3] = gamma_1..gamma_4, G[4] = gamma_5 */
static int g_ready = 0;

static void init_gamma(void)
{
    if (g_ready) return;
    cplx sig[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    memset(G, 0, sizeof(G));
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                G[k][a][2 + b] = -I * sig[k][a][b];
                G[k][2 + a][b] = I * sig[k][a][b];
            }
    for (int a = 0; a < 2; ++a) {
        G[3][a][2 + a] = 1;
        G[3][2 + a][a] = 1;
    }
    /* gamma_5 as the product g1 g2 g3 g4 (checked to be diag(1,1,-1,-1) by the tests) */
    cplx t1[4][4], t2[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += G[0][i][k] * G[1][k][j];
            t1[i][j] = s;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += t1[i][k] * G[2][k][j];
            t2[i][j] = s;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += t2[i][k] * G[3][k][j];
            G[4][i][j] = s;
        }
    g_ready = 1;
}

/* gamma matrix mu (0..3 = gamma_1..gamma_4, 4 = gamma_5), row-major 4x4 */
void or_gamma(int mu, cplx *out)
{
    init_gamma();
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) out[4 * i + j] = G[mu][i][j];
}

/* ------------------------------------------------------------------ */
/* lattice helpers                                                      */
/* ------------------------------------------------------------------ */
static long volume(const int *d) { return (long)d[0] * d[1] * d[2] * d[3]; }

static void coords(const int *d, long n, int c[4])
{
    c[0] = (int)(n % d[0]);
    n /= d[0];
    c[1] = (int)(n % d[1]);
    n /= d[1];
    c[2] = (int)(n % d[2]);
    c[3] = (int)(n / d[2]);
}

static long index_of(const int *d, const int c[4])
{
    return ((long)(c[3] * d[2] + c[2]) * d[1] + c[1]) * d[0] + c[0];
}

/* neighbour n + step*mu_hat (step = +1 or -1) and the boundary phase of the hop */
static long neighbour(const int *d, const double *bc, long n, int mu, int step, double *phase)
{
    int c[4];
    coords(d, n, c);
    *phase = 1.0;
    c[mu] += step;
    if (c[mu] == d[mu]) {
        c[mu] = 0;
        *phase = bc[mu];
    } else if (c[mu] < 0) {
        c[mu] = d[mu] - 1;
        *phase = bc[mu];
    }
    return index_of(d, c);
}

/* ------------------------------------------------------------------ */
/* Wilson operator, Eqs. (1)-(2)                                        */
/* ------------------------------------------------------------------ */
/* (T_mu psi)_n for one site, accumulated into acc[4][3]:
 *   mu > 0 : U_mu(n)            (1 - gamma_mu) psi_{n+mu}
 *   mu < 0 : U_mu(n-mu)^dagger  (1 + gamma_mu) psi_{n-mu}
 * The spin matrix acts on the spin index, the link on the colour index. */
static void hop_site(const int *d, const double *bc, const cplx *U, const cplx *in, long n,
                     cplx acc[4][3])
{
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) acc[s][a] = 0;
    for (int mu = 0; mu < 4; ++mu) {
        for (int dir = 0; dir < 2; ++dir) {
            int step = dir == 0 ? +1 : -1;
            double ph;
            long m = neighbour(d, bc, n, mu, step, &ph);
            /* spin matrix 1 -/+ gamma_mu */
            cplx P[4][4];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    P[i][j] = (i == j ? 1.0 : 0.0) - (double)step * G[mu][i][j];
            /* link: U_mu(n) forward, U_mu(n-mu)^dagger backward */
            cplx L[3][3];
            const cplx *u = step > 0 ? U + (n * 4 + mu) * 9 : U + (m * 4 + mu) * 9;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) L[a][b] = step > 0 ? u[3 * a + b] : conj(u[3 * b + a]);
            const cplx *p = in + m * 12;
            for (int s = 0; s < 4; ++s) {
                cplx chi[3];
                for (int b = 0; b < 3; ++b) {
                    cplx v = 0;
                    for (int t = 0; t < 4; ++t) v += P[s][t] * p[3 * t + b];
                    chi[b] = v;
                }
                for (int a = 0; a < 3; ++a) {
                    cplx v = 0;
                    for (int b = 0; b < 3; ++b) v += L[a][b] * chi[b];
                    acc[s][a] += ph * v;
                }
            }
        }
    }
}

/* out = D_w(m) in = (m + 4) in - 1/2 sum_{mu=+-1..+-4} T_mu in       (Eq. 1) */
void or_dslash(const int *d, const double *bc, const cplx *U, double m, const cplx *in, cplx *out)
{
    init_gamma();
    long V = volume(d);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; ++n) {
        cplx acc[4][3];
        hop_site(d, bc, U, in, n, acc);
        for (int s = 0; s < 4; ++s)
            for (int a = 0; a < 3; ++a)
                out[n * 12 + 3 * s + a] = (m + 4.0) * in[n * 12 + 3 * s + a] - 0.5 * acc[s][a];
    }
}

/* D_w(m) in at a list of sites only: out[k][12] = (D_w in)(sites[k]) */
void or_dslash_sites(const int *d, const double *bc, const cplx *U, double m, const cplx *in,
                     long nsites, const long *sites, cplx *out)
{
    init_gamma();
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nsites; ++k) {
        long n = sites[k];
        cplx acc[4][3];
        hop_site(d, bc, U, in, n, acc);
        for (int s = 0; s < 4; ++s)
            for (int a = 0; a < 3; ++a)
                out[k * 12 + 3 * s + a] = (m + 4.0) * in[n * 12 + 3 * s + a] - 0.5 * acc[s][a];
    }
}

/* out = gamma_5 in, by the explicit 4x4 matrix */
void or_gamma5(long nsites, const cplx *in, cplx *out)
{
    init_gamma();
#pragma omp parallel for schedule(static)
    for (long n = 0; n < nsites; ++n) {
        cplx tmp[12];
        for (int s = 0; s < 4; ++s)
            for (int a = 0; a < 3; ++a) {
                cplx v = 0;
                for (int t = 0; t < 4; ++t) v += G[4][s][t] * in[n * 12 + 3 * t + a];
                tmp[3 * s + a] = v;
            }
        memcpy(out + n * 12, tmp, sizeof(tmp));
    }
}

/* H_w = gamma_5 D_w(m)   (Sec. II: H_w is hermitian by gamma_5-hermiticity) */
void or_hw(const int *d, const double *bc, const cplx *U, double m, const cplx *in, cplx *out)
{
    or_dslash(d, bc, U, m, in, out);
    or_gamma5(volume(d), out, out);
}

/* ------------------------------------------------------------------ */
/* level-1 vector helpers (plain loops)                                 */
/* ------------------------------------------------------------------ */
static cplx vdot(long N, const cplx *a, const cplx *b) /* a^dagger b */
{
    double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (long i = 0; i < N; ++i) {
        cplx v = conj(a[i]) * b[i];
        re += creal(v);
        im += cimag(v);
    }
    return re + I * im;
}

static double vnorm2(long N, const cplx *a) { return creal(vdot(N, a, a)); }

/* ------------------------------------------------------------------ */
/* polynomial approximation P(x) ~ x^{-1/2} on [eps, 1], Eq. (4)        */
/* ------------------------------------------------------------------ */
/* Coefficients of the degree-n Chebyshev interpolant of x^{-1/2} on
 * [eps, 1] in the variable y = (2x - (1+eps)) / (1-eps):
 *   P(x) = sum_{k=0}^{n} c_k T_k(y),
 * interpolating at the n+1 Chebyshev nodes y_j = cos(pi (j+1/2)/(n+1)).
 * c[0] is returned already halved, so the sum above is plain. */
void or_cheb_coeffs(double eps, int n, double *c)
{
    int np = n + 1;
    double *f = malloc(sizeof(double) * np);
    for (int j = 0; j < np; ++j) {
        double th = M_PI * (j + 0.5) / np;
        double x = 0.5 * (1.0 + eps) + 0.5 * (1.0 - eps) * cos(th);
        f[j] = 1.0 / sqrt(x);
    }
    for (int k = 0; k <= n; ++k) {
        double s = 0;
        for (int j = 0; j < np; ++j) s += f[j] * cos(k * M_PI * (j + 0.5) / np);
        c[k] = 2.0 * s / np;
    }
    c[0] *= 0.5;
    free(f);
}

/* P(x) by Clenshaw's recurrence (the scalar form of Sec. V's recursion) */
double or_poly_eval(const double *c, int n, double eps, double x)
{
    double y = (2.0 * x - (1.0 + eps)) / (1.0 - eps);
    double b1 = 0, b2 = 0;
    for (int k = n; k >= 1; --k) {
        double b0 = c[k] + 2.0 * y * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return c[0] + y * b1 - b2;
}

/* delta = max_{x in [eps,1]} |1 - sqrt(x) P(x)| on npts log-spaced points (Eq. 4) */
double or_poly_delta(const double *c, int n, double eps, int npts)
{
    double dmax = 0;
    for (int i = 0; i < npts; ++i) {
        double x = exp(log(eps) + (log(1.0) - log(eps)) * i / (double)(npts - 1));
        double e = fabs(1.0 - sqrt(x) * or_poly_eval(c, n, eps, x));
        if (e > dmax) dmax = e;
    }
    return dmax;
}

/* ------------------------------------------------------------------ */
/* sign(H_w) with low-mode deflation, Eqs. (5)-(7)                      */
/* ------------------------------------------------------------------ */
typedef struct {
    const int *d;
    const double *bc;
    const cplx *U;
    double mw;      /* Wilson mass inside H_w */
    double lmax;    /* ||H_w|| estimate: Q = H_w / lmax */
    double eps;
    int n;
    const double *c;
    int nev;
    const double *lam; /* eigenvalues of H_w (signed) */
    const cplx *eta;   /* eigenvectors [nev][12V], orthonormal */
    /* rational form of Eq. (12) instead of the polynomial when npoles > 0:
       P(Q^2) psi_h = sum_i rb_i (Q^2 + rc_i)^-1 psi_h, solved by multi-shift CG to rtol */
    int npoles;
    const double *rb, *rc;
    double rtol;
} sign_args;

/* out = Y in, with Y = (2 Q^2 - (1+eps)) / (1-eps), Q = H_w / lmax */
static void apply_Y(const sign_args *a, const cplx *in, cplx *out, cplx *tmp)
{
    long N = 12 * volume(a->d);
    or_hw(a->d, a->bc, a->U, a->mw, in, tmp);
    or_hw(a->d, a->bc, a->U, a->mw, tmp, out);
    double s = 2.0 / (a->lmax * a->lmax * (1.0 - a->eps));
    double t = (1.0 + a->eps) / (1.0 - a->eps);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) out[i] = s * out[i] - t * in[i];
}

static void rational_apply(const sign_args *a, const cplx *ph, cplx *pp);

/* sign(H_w) in ~ sum_i sign(lam_i) (eta_i^dag in) eta_i + Q P(Q^2) (1 - P_l) in   (Eq. 7) */
static void sign_apply(const sign_args *a, const cplx *in, cplx *out)
{
    long N = 12 * volume(a->d);
    cplx *ph = malloc(sizeof(cplx) * N);
    cplx *b1 = calloc(N, sizeof(cplx));
    cplx *b2 = calloc(N, sizeof(cplx));
    cplx *y = malloc(sizeof(cplx) * N);
    cplx *tmp = malloc(sizeof(cplx) * N);
    cplx *proj = malloc(sizeof(cplx) * (a->nev > 0 ? a->nev : 1));

    /* psi_h = psi - sum_i eta_i (eta_i^dag psi)    (Eq. 6) */
    memcpy(ph, in, sizeof(cplx) * N);
    for (int i = 0; i < a->nev; ++i) {
        const cplx *e = a->eta + (long)i * N;
        proj[i] = vdot(N, e, in);
        for (long k = 0; k < N; ++k) ph[k] -= proj[i] * e[k];
    }

    cplx *pp = y; /* P(Q^2) psi_h */
    if (a->npoles > 0) {
        rational_apply(a, ph, pp); /* Eq. (12) */
        goto outer;
    }
    /* Clenshaw: b_k = c_k psi_h + 2 Y b_{k+1} - b_{k+2}, k = n..1;
       P psi_h = c_0 psi_h + Y b_1 - b_2                            (Sec. V) */
    for (long k = 0; k < N; ++k) b1[k] = a->c[a->n] * ph[k]; /* b_n (b_{n+1} = 0) */
    for (int k = a->n - 1; k >= 1; --k) {
        apply_Y(a, b1, y, tmp);
        for (long i = 0; i < N; ++i) {
            cplx b0 = a->c[k] * ph[i] + 2.0 * y[i] - b2[i];
            b2[i] = b1[i];
            b1[i] = b0;
        }
    }
    if (a->n >= 1) {
        apply_Y(a, b1, y, tmp);
        for (long i = 0; i < N; ++i) pp[i] = a->c[0] * ph[i] + y[i] - b2[i];
    } else {
        for (long i = 0; i < N; ++i) pp[i] = a->c[0] * ph[i];
    }
outer:
    /* Q P(Q^2) psi_h */
    or_hw(a->d, a->bc, a->U, a->mw, pp, out);
    for (long i = 0; i < N; ++i) out[i] /= a->lmax;
    /* + sum_i sign(lam_i) (eta_i^dag psi) eta_i */
    for (int i = 0; i < a->nev; ++i) {
        const cplx *e = a->eta + (long)i * N;
        double sg = a->lam[i] > 0 ? 1.0 : (a->lam[i] < 0 ? -1.0 : 0.0);
        for (long k = 0; k < N; ++k) out[k] += sg * proj[i] * e[k];
    }
    free(ph);
    free(b1);
    free(b2);
    free(y);
    free(tmp);
    free(proj);
}

/* out = sign(H_w(mw)) in (approximated by Eq. 7) */
void or_sign(const int *d, const double *bc, const cplx *U, double mw, double lmax, double eps,
             int n, const double *c, int nev, const double *lam, const cplx *eta, const cplx *in,
             cplx *out)
{
    init_gamma();
    sign_args a = {d, bc, U, mw, lmax, eps, n, c, nev, lam, eta};
    sign_apply(&a, in, out);
}

/* ------------------------------------------------------------------ */
/* Lanczos on H_w^2: the rescale lambda_max (Eq. 5) and the low modes   */
/* (Eq. 7), Sec. V's eigensolver of H_w in its plainest form           */
/* ------------------------------------------------------------------ */
/* Eigen-decomposition of an n x n Hermitian matrix A (row major, destroyed) by
 * cyclic Jacobi rotations: ev ascending, Z[k*n + i] = component k of eigenvector i. */
static void herm_jacobi(int n, cplx *A, double *ev, cplx *Z)
{
    for (int i = 0; i < n * n; ++i) Z[i] = 0;
    for (int i = 0; i < n; ++i) Z[i * n + i] = 1;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double a = creal(A[i * n + j] * conj(A[i * n + j]));
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const cplx apq = A[p * n + q];
                const double b = cabs(apq);
                if (b == 0.0) continue;
                /* rotate in the (p, q) plane: with u = apq / |apq|, the 2x2 block
                   [[a, b u], [b conj(u), d]] is diagonalised by c, s with t = s / c solving
                   t^2 + 2 zeta t - 1 = 0, zeta = (d - a) / (2 b) */
                const double a = creal(A[p * n + p]), d = creal(A[q * n + q]);
                const cplx u = apq / b;
                const double zeta = (d - a) / (2.0 * b);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(zeta * zeta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* columns p, q */
                    const cplx akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * conj(u) * akq;
                    A[k * n + q] = s * u * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* rows p, q */
                    const cplx apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * u * aqk;
                    A[q * n + k] = s * conj(u) * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const cplx zkp = Z[k * n + p], zkq = Z[k * n + q];
                    Z[k * n + p] = c * zkp - s * conj(u) * zkq;
                    Z[k * n + q] = s * u * zkp + c * zkq;
                }
            }
    }
    /* sort ascending (selection sort on the diagonal, columns of Z follow) */
    for (int i = 0; i < n; ++i) ev[i] = creal(A[i * n + i]);
    for (int i = 0; i < n; ++i) {
        int m = i;
        for (int j = i + 1; j < n; ++j)
            if (ev[j] < ev[m]) m = j;
        if (m != i) {
            double t = ev[i];
            ev[i] = ev[m];
            ev[m] = t;
            for (int k = 0; k < n; ++k) {
                cplx z = Z[k * n + i];
                Z[k * n + i] = Z[k * n + m];
                Z[k * n + m] = z;
            }
        }
    }
}

/* m-step Lanczos on H_w(mw)^2 from the start vector v0, with full re-orthogonalisation (classical
 * Gram-Schmidt, twice), keeping the basis V [m][12V].  Returns the number of steps taken (fewer when
 * the Krylov space closes). */
static int lanczos_basis(const int *d, const double *bc, const cplx *U, double mw, int m, const cplx *v0, cplx *V)
{
    long N = 12 * volume(d);
    cplx *w = malloc(sizeof(cplx) * N), *t = malloc(sizeof(cplx) * N);
    double nr = sqrt(vnorm2(N, v0));
    for (long k = 0; k < N; ++k) V[k] = v0[k] / nr;
    int steps = m;
    for (int j = 0; j < m; ++j) {
        or_hw(d, bc, U, mw, V + (long)j * N, t);
        or_hw(d, bc, U, mw, t, w);
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i <= j; ++i) {
                const cplx *vi = V + (long)i * N;
                cplx h = vdot(N, vi, w);
                for (long k = 0; k < N; ++k) w[k] -= h * vi[k];
            }
        double beta = sqrt(vnorm2(N, w));
        if (j + 1 == m) break;
        if (beta < 1e-13) {
            steps = j + 1;
            break;
        }
        for (long k = 0; k < N; ++k) V[(long)(j + 1) * N + k] = w[k] / beta;
    }
    free(w);
    free(t);
    return steps;
}

/* lambda_max estimate (Sec. II rescale, Eq. 5): the square root of the largest Ritz value of H_w^2
 * from `steps` Lanczos steps started from v0 (a lower bound of the largest |eigenvalue| of H_w). */
double or_lambda_max(const int *d, const double *bc, const cplx *U, double mw, int steps, const cplx *v0)
{
    init_gamma();
    long N = 12 * volume(d);
    cplx *V = malloc(sizeof(cplx) * N * steps), *w = malloc(sizeof(cplx) * N), *t = malloc(sizeof(cplx) * N);
    int m = lanczos_basis(d, bc, U, mw, steps, v0, V);
    /* Rayleigh-Ritz of H_w^2 in the basis: T_ij = v_i^dag H_w^2 v_j */
    cplx *T = malloc(sizeof(cplx) * m * m), *Z = malloc(sizeof(cplx) * m * m);
    double *ev = malloc(sizeof(double) * m);
    for (int j = 0; j < m; ++j) {
        or_hw(d, bc, U, mw, V + (long)j * N, t);
        or_hw(d, bc, U, mw, t, w);
        for (int i = 0; i < m; ++i) T[i * m + j] = vdot(N, V + (long)i * N, w);
    }
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j) {
            cplx a = 0.5 * (T[i * m + j] + conj(T[j * m + i]));
            T[i * m + j] = a;
            T[j * m + i] = conj(a);
        }
    herm_jacobi(m, T, ev, Z);
    double top = sqrt(ev[m - 1] > 0 ? ev[m - 1] : 0.0);
    free(V);
    free(w);
    free(t);
    free(T);
    free(Z);
    free(ev);
    return top;
}

/* Rayleigh-Ritz of the Hermitian operator op on the orthonormal basis B [k][12V]: the k x k matrix
 * B^dag op B, its eigenpairs (ascending) and the Ritz vectors out [k][12V] */
static void rayleigh_ritz(const int *d, const double *bc, const cplx *U, double mw, int squared, int k,
                          const cplx *B, double *ev, cplx *out)
{
    long N = 12 * volume(d);
    cplx *w = malloc(sizeof(cplx) * N), *t = malloc(sizeof(cplx) * N);
    cplx *T = malloc(sizeof(cplx) * k * k), *Z = malloc(sizeof(cplx) * k * k);
    for (int j = 0; j < k; ++j) {
        if (squared) {
            or_hw(d, bc, U, mw, B + (long)j * N, t);
            or_hw(d, bc, U, mw, t, w);
        } else {
            or_hw(d, bc, U, mw, B + (long)j * N, w);
        }
        for (int i = 0; i < k; ++i) T[i * k + j] = vdot(N, B + (long)i * N, w);
    }
    for (int i = 0; i < k; ++i)
        for (int j = i; j < k; ++j) {
            cplx a = 0.5 * (T[i * k + j] + conj(T[j * k + i]));
            T[i * k + j] = a;
            T[j * k + i] = conj(a);
        }
    herm_jacobi(k, T, ev, Z);
    for (int i = 0; i < k; ++i) {
        cplx *e = out + (long)i * N;
        for (long q = 0; q < N; ++q) e[q] = 0;
        for (int j = 0; j < k; ++j) {
            const cplx z = Z[j * k + i];
            const cplx *bj = B + (long)j * N;
            for (long q = 0; q < N; ++q) e[q] += z * bj[q];
        }
    }
    free(w);
    free(t);
    free(T);
    free(Z);
}

/* The nev eigenpairs of H_w with smallest |lambda| (Sec. V: eigenvectors of H_w from a Krylov space of
 * H_w^2): m Lanczos steps on H_w^2 from v0; Rayleigh-Ritz with H_w^2 on the basis (its smallest Ritz
 * values are extremes of H_w^2, so they converge without spurious interior values); then Rayleigh-Ritz
 * with H_w itself on the nev + 8 smallest of those Ritz vectors (a span that holds both partners of
 * every +-lambda pair), which gives the signed lambda of Eq. 7.  vals [nev], vecs [nev][12V], sorted by
 * |lambda|; returns the largest eigen-residual |H_w eta - lambda eta| of the returned pairs. */
double or_lanczos_lowmodes(const int *d, const double *bc, const cplx *U, double mw, int m, int nev, const cplx *v0,
                           double *vals, cplx *vecs)
{
    init_gamma();
    long N = 12 * volume(d);
    cplx *V = malloc(sizeof(cplx) * N * m), *w = malloc(sizeof(cplx) * N);
    int mm = lanczos_basis(d, bc, U, mw, m, v0, V);
    cplx *R2 = malloc(sizeof(cplx) * N * mm);
    double *ev2 = malloc(sizeof(double) * mm);
    rayleigh_ritz(d, bc, U, mw, 1, mm, V, ev2, R2);
    int k = nev + 8 < mm ? nev + 8 : mm;
    cplx *R1 = malloc(sizeof(cplx) * N * k);
    double *ev1 = malloc(sizeof(double) * k);
    rayleigh_ritz(d, bc, U, mw, 0, k, R2, ev1, R1);
    int *o = malloc(sizeof(int) * k);
    for (int i = 0; i < k; ++i) o[i] = i;
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j)
            if (fabs(ev1[o[j]]) < fabs(ev1[o[i]])) {
                int t = o[i];
                o[i] = o[j];
                o[j] = t;
            }
    double worst = 0;
    for (int q = 0; q < nev && q < k; ++q) {
        vals[q] = ev1[o[q]];
        memcpy(vecs + (long)q * N, R1 + (long)o[q] * N, sizeof(cplx) * N);
        or_hw(d, bc, U, mw, vecs + (long)q * N, w);
        for (long i = 0; i < N; ++i) w[i] -= vals[q] * vecs[(long)q * N + i];
        double r = sqrt(vnorm2(N, w));
        if (r > worst) worst = r;
    }
    free(o);
    free(V);
    free(w);
    free(R2);
    free(ev2);
    free(R1);
    free(ev1);
    return worst;
}

/* ------------------------------------------------------------------ */
/* rational approximation, Eq. (12): Zolotarev's optimal P(x) ~ x^-1/2  */
/* ------------------------------------------------------------------ */
/* Complete elliptic integral K(m) of parameter m = k^2 (k the modulus), by the
 * arithmetic-geometric mean: K = pi / (2 AGM(1, sqrt(1 - m))). */
double or_ellipk(double m)
{
    double a = 1.0, b = sqrt(1.0 - m);
    for (int i = 0; i < 60 && fabs(a - b) > 1e-16 * a; ++i) {
        double an = 0.5 * (a + b);
        b = sqrt(a * b);
        a = an;
    }
    return M_PI / (2.0 * a);
}

/* Jacobi elliptic functions sn, cn, dn of argument u and parameter m, by the
 * descending AGM (Abramowitz and Stegun 16.4.3): a_0 = 1, b_0 = sqrt(1-m),
 * c_0 = sqrt(m); phi_N = 2^N a_N u; phi_{j-1} = (phi_j + asin(c_j sin(phi_j) / a_j)) / 2;
 * sn = sin(phi_0), cn = cos(phi_0), dn = cn / cos(phi_1 - phi_0). */
void or_jacobi(double u, double m, double *sn, double *cn, double *dn)
{
    double a[64], c[64];
    a[0] = 1.0;
    double b = sqrt(1.0 - m);
    c[0] = sqrt(m);
    int N = 0;
    while (N < 62 && fabs(c[N]) > 1e-16) {
        a[N + 1] = 0.5 * (a[N] + b);
        c[N + 1] = 0.5 * (a[N] - b);
        b = sqrt(a[N] * b);
        ++N;
    }
    double phi = ldexp(1.0, N) * a[N] * u, phi1 = phi;
    for (int j = N; j >= 1; --j) {
        phi1 = phi;
        phi = 0.5 * (phi + asin(c[j] * sin(phi) / a[j]));
    }
    *sn = sin(phi);
    *cn = cos(phi);
    *dn = N ? *cn / cos(phi1 - phi) : 1.0;
}

/* Zolotarev's optimal rational approximation of type (2n-1, 2n) to sign(q) on
 * k <= |q| <= 1 (k = sqrt(eps)): sign(q) ~ D q prod_{j<n} (q^2 + a_{2j}) / prod_{i<=n} (q^2 + a_{2i-1}),
 * a_l = eps sn^2(l K'/(2n); 1-eps) / cn^2(l K'/(2n); 1-eps), K' = K(1-eps).  As P(x) ~ x^-1/2
 * on [eps, 1] (x = q^2) in partial fractions (the form of Eq. 12):
 *   P(x) = sum_{i=1}^{n} b_i / (x + c_i),  c_i = a_{2i-1},
 *   b_i = D prod_j (a_{2j} - c_i) / prod_{l != i} (c_l - c_i).
 * D puts the error 1 - sqrt(x) P(x) in equioscillation: D = 2 / (max f + min f) for
 * f(q) = q prod / prod on [k, 1], its extremes located on a grid and refined by golden
 * section.  Returns delta = (max f - min f) / (max f + min f) (Eq. 4). */
static double zolo_f(int n, const double *a, double q)
{
    double v = q;
    for (int j = 1; j < n; ++j) v *= q * q + a[2 * j];
    for (int i = 1; i <= n; ++i) v /= q * q + a[2 * i - 1];
    return v;
}

static double golden_extreme(int n, const double *a, double lo, double hi, int maximise)
{
    const double g = 0.5 * (sqrt(5.0) - 1.0);
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    double f1 = zolo_f(n, a, x1), f2 = zolo_f(n, a, x2);
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        if ((f1 > f2) == (maximise != 0)) {
            hi = x2;
            x2 = x1;
            f2 = f1;
            x1 = hi - g * (hi - lo);
            f1 = zolo_f(n, a, x1);
        } else {
            lo = x1;
            x1 = x2;
            f1 = f2;
            x2 = lo + g * (hi - lo);
            f2 = zolo_f(n, a, x2);
        }
    }
    return zolo_f(n, a, 0.5 * (lo + hi));
}

double or_zolotarev(double eps, int n, double *b, double *c)
{
    double *a = malloc(sizeof(double) * (2 * n + 1));
    const double m = 1.0 - eps, Kp = or_ellipk(m);
    for (int l = 1; l <= 2 * n - 1; ++l) {
        double sn, cn, dn;
        or_jacobi(l * Kp / (2.0 * n), m, &sn, &cn, &dn);
        a[l] = eps * sn * sn / (cn * cn);
    }
    /* extremes of f on [k, 1]: the end points and the interior local extremes */
    const double k = sqrt(eps);
    const int G = 20000;
    double fhi = fmax(zolo_f(n, a, k), zolo_f(n, a, 1.0)), flo = fmin(zolo_f(n, a, k), zolo_f(n, a, 1.0));
    double qp = k, fp = zolo_f(n, a, k);
    double qc = exp(log(k) * (1.0 - 1.0 / G)), fc = zolo_f(n, a, qc);
    for (int i = 2; i <= G; ++i) {
        double qn = exp(log(k) * (1.0 - (double)i / G)), fn = zolo_f(n, a, qn);
        if (fc > fp && fc >= fn) fhi = fmax(fhi, golden_extreme(n, a, qp, qn, 1));
        if (fc < fp && fc <= fn) flo = fmin(flo, golden_extreme(n, a, qp, qn, 0));
        qp = qc;
        fp = fc;
        qc = qn;
        fc = fn;
    }
    const double D = 2.0 / (fhi + flo);
    for (int i = 1; i <= n; ++i) {
        const double ci = a[2 * i - 1];
        double v = D;
        for (int j = 1; j < n; ++j) v *= a[2 * j] - ci;
        for (int l = 1; l <= n; ++l)
            if (l != i) v /= a[2 * l - 1] - ci;
        c[i - 1] = ci;
        b[i - 1] = v;
    }
    free(a);
    return (fhi - flo) / (fhi + flo);
}

/* P(x) = sum_i b_i / (x + c_i) */
double or_rational_eval(const double *b, const double *c, int n, double x)
{
    double v = 0;
    for (int i = 0; i < n; ++i) v += b[i] / (x + c[i]);
    return v;
}

/* pp = sum_i rb_i (Q^2 + rc_i)^-1 ph by one multi-shift CG (Eq. 12 and the
 * multi-shifted CG of Sec. V): CG on the base system (Q^2 + c_0) x = ph, c_0 the smallest
 * shift, the others (Q^2 + c_0 + s_i) x_i = ph with s_i = c_i - c_0 >= 0 from the same Krylov
 * space (collinear residuals r_i = z_i r, the shifted-system recurrences of Jegerlehner 1996);
 * each shift stops updating once |z_i| |r| <= rtol |ph|. */
static void rational_apply(const sign_args *a, const cplx *ph, cplx *pp)
{
    long N = 12 * volume(a->d);
    const int n = a->npoles;
    int i0 = 0;
    for (int i = 1; i < n; ++i)
        if (a->rc[i] < a->rc[i0]) i0 = i;
    const double c0 = a->rc[i0];
    cplx *r = malloc(sizeof(cplx) * N), *p = malloc(sizeof(cplx) * N), *q = malloc(sizeof(cplx) * N);
    cplx *tmp = malloc(sizeof(cplx) * N), *ps = malloc(sizeof(cplx) * N * n), *xs = calloc((size_t)N * n, sizeof(cplx));
    double *z = malloc(sizeof(double) * n), *zo = malloc(sizeof(double) * n), *zn = malloc(sizeof(double) * n);
    int *act = malloc(sizeof(int) * n);
    memcpy(r, ph, sizeof(cplx) * N);
    memcpy(p, ph, sizeof(cplx) * N);
    for (int i = 0; i < n; ++i) {
        memcpy(ps + (long)i * N, ph, sizeof(cplx) * N);
        z[i] = zo[i] = 1.0;
        act[i] = 1;
    }
    const double bn = sqrt(vnorm2(N, ph));
    double rr = bn * bn, alpha_o = 1.0, beta_o = 0.0;
    const double s2 = 1.0 / (a->lmax * a->lmax);
    for (int it = 0; it < 100000 && bn > 0; ++it) {
        int any = 0;
        for (int i = 0; i < n; ++i) any |= act[i];
        if (!any) break;
        /* q = (Q^2 + c_0) p */
        or_hw(a->d, a->bc, a->U, a->mw, p, tmp);
        or_hw(a->d, a->bc, a->U, a->mw, tmp, q);
        for (long k = 0; k < N; ++k) q[k] = s2 * q[k] + c0 * p[k];
        const double alpha = rr / creal(vdot(N, p, q));
        for (int i = 0; i < n; ++i) {
            zn[i] = z[i];
            if (!act[i]) continue;
            const double si = a->rc[i] - c0;
            zn[i] = z[i] * zo[i] * alpha_o / (alpha * beta_o * (zo[i] - z[i]) + zo[i] * alpha_o * (1.0 + si * alpha));
            const double ai = alpha * zn[i] / z[i];
            cplx *xi = xs + (long)i * N, *pi = ps + (long)i * N;
            for (long k = 0; k < N; ++k) xi[k] += ai * pi[k];
        }
        for (long k = 0; k < N; ++k) r[k] -= alpha * q[k];
        const double rn = vnorm2(N, r), beta = rn / rr;
        for (int i = 0; i < n; ++i) {
            if (act[i]) {
                const double bi = beta * (zn[i] / z[i]) * (zn[i] / z[i]);
                cplx *pi = ps + (long)i * N;
                for (long k = 0; k < N; ++k) pi[k] = zn[i] * r[k] + bi * pi[k];
                if (fabs(zn[i]) * sqrt(rn) <= a->rtol * bn) act[i] = 0;
            }
            if (zn[i] != z[i]) {
                zo[i] = z[i];
                z[i] = zn[i];
            }
        }
        for (long k = 0; k < N; ++k) p[k] = r[k] + beta * p[k];
        alpha_o = alpha;
        beta_o = beta;
        rr = rn;
    }
    memset(pp, 0, sizeof(cplx) * N);
    for (int i = 0; i < n; ++i)
        for (long k = 0; k < N; ++k) pp[k] += a->rb[i] * xs[(long)i * N + k];
    free(r);
    free(p);
    free(q);
    free(tmp);
    free(ps);
    free(xs);
    free(z);
    free(zo);
    free(zn);
    free(act);
}

/* out = sign(H_w(mw)) in with the rational P of Eq. (12) (partial fractions rb, rc) */
void or_sign_rational(const int *d, const double *bc, const cplx *U, double mw, double lmax, int npoles,
                      const double *rb, const double *rc, double rtol, int nev, const double *lam, const cplx *eta,
                      const cplx *in, cplx *out)
{
    init_gamma();
    sign_args a = {d, bc, U, mw, lmax, 0.0, 0, NULL, nev, lam, eta, npoles, rb, rc, rtol};
    sign_apply(&a, in, out);
}

/* D(m) in with the rational sign (Eqs. 3, 8, 12) */
void or_overlap_rational(const int *d, const double *bc, const cplx *U, double rho, double mass, double lmax,
                         int npoles, const double *rb, const double *rc, double rtol, int nev, const double *lam,
                         const cplx *eta, const cplx *in, cplx *out)
{
    init_gamma();
    long V = volume(d), N = 12 * V;
    sign_args a = {d, bc, U, -rho, lmax, 0.0, 0, NULL, nev, lam, eta, npoles, rb, rc, rtol};
    cplx *s = malloc(sizeof(cplx) * N);
    sign_apply(&a, in, s);
    or_gamma5(V, s, s);
    for (long i = 0; i < N; ++i) {
        cplx Dpsi = in[i] + s[i];
        out[i] = rho * Dpsi + mass * (in[i] - 0.5 * Dpsi);
    }
    free(s);
}

/* ------------------------------------------------------------------ */
/* overlap operator, Eqs. (3) and (8)                                   */
/* ------------------------------------------------------------------ */
/* D psi = psi + gamma_5 sign(H_w(-rho)) psi   (massless, Eq. 3)
 * D(m) psi = rho D psi + m (1 - D/2) psi     (Eq. 8, lattice spacing a = 1) */
void or_overlap(const int *d, const double *bc, const cplx *U, double rho, double mass, double lmax,
                double eps, int n, const double *c, int nev, const double *lam, const cplx *eta,
                const cplx *in, cplx *out)
{
    init_gamma();
    long V = volume(d), N = 12 * V;
    sign_args a = {d, bc, U, -rho, lmax, eps, n, c, nev, lam, eta};
    cplx *s = malloc(sizeof(cplx) * N);
    sign_apply(&a, in, s);
    or_gamma5(V, s, s);
    for (long i = 0; i < N; ++i) {
        cplx Dpsi = in[i] + s[i];
        out[i] = rho * Dpsi + mass * (in[i] - 0.5 * Dpsi);
    }
    free(s);
}

/* D(m)^dagger D(m) psi = gamma_5 D(m) gamma_5 D(m) psi (gamma_5-hermiticity of D) */
static void ddag_d(const sign_args *a, double rho, double mass, const cplx *in, cplx *out, cplx *t)
{
    long V = volume(a->d), N = 12 * V;
    cplx *s = malloc(sizeof(cplx) * N);
    /* t = D(m) in */
    sign_apply(a, in, s);
    or_gamma5(V, s, s);
    for (long i = 0; i < N; ++i) {
        cplx Dpsi = in[i] + s[i];
        t[i] = rho * Dpsi + mass * (in[i] - 0.5 * Dpsi);
    }
    /* out = gamma_5 D(m) gamma_5 t */
    or_gamma5(V, t, t);
    sign_apply(a, t, s);
    or_gamma5(V, s, s);
    for (long i = 0; i < N; ++i) {
        cplx Dpsi = t[i] + s[i];
        out[i] = rho * Dpsi + mass * (t[i] - 0.5 * Dpsi);
    }
    or_gamma5(V, out, out);
    free(s);
}

void or_overlap_normal(const int *d, const double *bc, const cplx *U, double rho, double mass,
                       double lmax, double eps, int n, const double *c, int nev, const double *lam,
                       const cplx *eta, const cplx *in, cplx *out)
{
    init_gamma();
    long N = 12 * volume(d);
    sign_args a = {d, bc, U, -rho, lmax, eps, n, c, nev, lam, eta};
    cplx *t = malloc(sizeof(cplx) * N);
    ddag_d(&a, rho, mass, in, out, t);
    free(t);
}

/* ------------------------------------------------------------------ */
/* deflated CG on D(m)^dagger D(m), Eq. (9) for the normal equations   */
/* ------------------------------------------------------------------ */
/* Solves A x = b, A = D(m)^dag D(m), to ||b - A x|| / ||b|| <= tol.
 * Deflation with nev2 eigenpairs (mu_i, xi_i) of A: every cycle forms the
 * true residual r = b - A x and solves its low part exactly,
 * x += sum_i xi_i (xi_i^dag r) / mu_i (pairs with mu_i <= zero_tol * mu_max
 * are excluded: exact zero modes, pseudo-inverse); CG then runs on the
 * orthogonal complement with the residual projected by
 * P_perp = 1 - sum_i xi_i xi_i^dag after every update, until the CG
 * residual meets tol; the next cycle checks the true residual.
 * Returns the number of CG iterations (negative if max_iter was reached);
 * *true_res gets the final ||b - A x|| / ||b||. */
int or_cg(const int *d, const double *bc, const cplx *U, double rho, double mass, double lmax,
          double eps, int n, const double *c, int nev, const double *lam, const cplx *eta, int nev2,
          const double *mu, const cplx *xi, double zero_tol, const cplx *b, cplx *x, double tol,
          int max_iter, double *true_res)
{
    init_gamma();
    long N = 12 * volume(d);
    sign_args a = {d, bc, U, -rho, lmax, eps, n, c, nev, lam, eta};
    cplx *r = malloc(sizeof(cplx) * N), *p = malloc(sizeof(cplx) * N);
    cplx *q = malloc(sizeof(cplx) * N), *t = malloc(sizeof(cplx) * N);
    double mu_max = 0;
    for (int i = 0; i < nev2; ++i)
        if (mu[i] > mu_max) mu_max = mu[i];
    double bnorm = sqrt(vnorm2(N, b));
    int iters = 0;

    memset(x, 0, sizeof(cplx) * N);
    double rel = 1.0;
    for (int cycle = 0; cycle < 20 && iters < max_iter; ++cycle) {
        /* r = b - A x */
        ddag_d(&a, rho, mass, x, q, t);
        for (long k = 0; k < N; ++k) r[k] = b[k] - q[k];
        rel = sqrt(vnorm2(N, r)) / bnorm;
        if (rel <= tol) break;
        /* low-mode part solved exactly on the current residual (Eq. 9):
           x += sum_i xi_i (xi_i^dag r) / mu_i, r <- P_perp r.  In the first cycle r = b
           and this is the deflated initial guess; later cycles remove what is left of
           the low-mode error when the xi_i are only approximate eigenvectors. */
        for (int i = 0; i < nev2; ++i) {
            const cplx *e = xi + (long)i * N;
            cplx pr = vdot(N, e, r);
            if (mu[i] > zero_tol * mu_max)
                for (long k = 0; k < N; ++k) x[k] += (pr / mu[i]) * e[k];
            for (long k = 0; k < N; ++k) r[k] -= pr * e[k];
        }
        memcpy(p, r, sizeof(cplx) * N);
        double rr = vnorm2(N, r);
        if (sqrt(rr) / bnorm <= tol) continue; /* the low-mode solve was enough */
        while (iters < max_iter) {
            ddag_d(&a, rho, mass, p, q, t);
            double pq = creal(vdot(N, p, q));
            double alpha = rr / pq;
            for (long k = 0; k < N; ++k) {
                x[k] += alpha * p[k];
                r[k] -= alpha * q[k];
            }
            for (int i = 0; i < nev2; ++i) {
                const cplx *e = xi + (long)i * N;
                cplx pr = vdot(N, e, r);
                for (long k = 0; k < N; ++k) r[k] -= pr * e[k];
            }
            double rr_new = vnorm2(N, r);
            ++iters;
            if (sqrt(rr_new) / bnorm <= tol) break;
            double beta = rr_new / rr;
            rr = rr_new;
            for (long k = 0; k < N; ++k) p[k] = r[k] + beta * p[k];
        }
    }
    ddag_d(&a, rho, mass, x, q, t);
    for (long k = 0; k < N; ++k) r[k] = b[k] - q[k];
    rel = sqrt(vnorm2(N, r)) / bnorm;
    *true_res = rel;
    free(r);
    free(p);
    free(q);
    free(t);
    return rel <= tol ? iters : -iters;
}

/* ------------------------------------------------------------------ */
/* multi-mass CG (Sec. II: one multi-shifted CG for several quark       */
/* masses, with the low modes of the massless D^dag D deflated)          */
/* ------------------------------------------------------------------ */
/* With sign^2 = 1, D(m)^dag D(m) = a_m (D^dag D + s_m), a_m = 1 - m^2/(4 rho^2),
 * s_m = m^2 / a_m (D = D(0) from Eq. 8; D^dag D = rho (D + D^dag)).  All masses
 * therefore share the Krylov space of D^dag D: the shifted systems
 * (D^dag D + s_k) y_k = b_h are solved by one CG recursion on D^dag D whose
 * shifted residuals are collinear with the base residual, r_k = z_k r, and
 * x_k = y_k / a_k + sum_i xi_i (xi_i^dag b) / (a_k mu_i + m_k^2) (Eq. 9).
 * The coefficient recurrences (z_k, alpha_k, beta_k) are those of the
 * shifted-system CG of Jegerlehner (1996), with base shift 0:
 *   z_k' = z_k z_k^- alpha^- / (alpha beta^- (z_k^- - z_k) + z_k^- alpha^- (1 + s_k alpha)),
 *   alpha_k = alpha z_k' / z_k,  beta_k = beta (z_k' / z_k)^2,  p_k <- z_k' r + beta_k p_k.
 * Each mass stops updating once |z_k| |r| <= tol |b_h|.  true_res[k] is the
 * relative residual of x_k with the full two-sign D(m_k)^dag D(m_k).
 * Returns the number of iterations. */
int or_multimass_cg(const int *d, const double *bc, const cplx *U, double rho, double lmax, double eps, int n,
                    const double *c, int nev, const double *lam, const cplx *eta, int nev2, const double *mu,
                    const cplx *xi, int nm, const double *masses, const cplx *b, cplx *x, double tol,
                    int max_iter, double *true_res)
{
    init_gamma();
    long N = 12 * volume(d);
    sign_args a = {d, bc, U, -rho, lmax, eps, n, c, nev, lam, eta};
    cplx *r = malloc(sizeof(cplx) * N), *p = malloc(sizeof(cplx) * N);
    cplx *q = malloc(sizeof(cplx) * N), *t = malloc(sizeof(cplx) * N);
    cplx *pk = malloc(sizeof(cplx) * N * nm);
    double *am = malloc(sizeof(double) * nm), *sm = malloc(sizeof(double) * nm);
    double *z = malloc(sizeof(double) * nm), *zo = malloc(sizeof(double) * nm);
    double *zn = malloc(sizeof(double) * nm);
    int *active = malloc(sizeof(int) * nm);
    for (int k = 0; k < nm; ++k) {
        am[k] = 1.0 - masses[k] * masses[k] / (4.0 * rho * rho);
        sm[k] = masses[k] * masses[k] / am[k];
        z[k] = zo[k] = 1.0;
        active[k] = 1;
    }
    /* b_h = b - sum_i xi_i (xi_i^dag b); low-mode coefficients kept for the end */
    memcpy(r, b, sizeof(cplx) * N);
    cplx *pb = malloc(sizeof(cplx) * (nev2 > 0 ? nev2 : 1));
    for (int i = 0; i < nev2; ++i) {
        const cplx *e = xi + (long)i * N;
        pb[i] = vdot(N, e, b);
        for (long k = 0; k < N; ++k) r[k] -= pb[i] * e[k];
    }
    double bh = sqrt(vnorm2(N, r));
    memset(x, 0, sizeof(cplx) * N * nm);
    memcpy(p, r, sizeof(cplx) * N);
    for (int k = 0; k < nm; ++k) memcpy(pk + (long)k * N, r, sizeof(cplx) * N);
    double rr = vnorm2(N, r), alpha_o = 1.0, beta_o = 0.0;
    int iters = 0;
    while (iters < max_iter && bh > 0) {
        int any = 0;
        for (int k = 0; k < nm; ++k) any |= active[k];
        if (!any) break;
        ddag_d(&a, rho, 0.0, p, q, t); /* massless D^dag D on the deflated complement */
        for (int i = 0; i < nev2; ++i) {
            const cplx *e = xi + (long)i * N;
            cplx pr = vdot(N, e, q);
            for (long k = 0; k < N; ++k) q[k] -= pr * e[k];
        }
        double alpha = rr / creal(vdot(N, p, q));
        for (int k = 0; k < nm; ++k) {
            zn[k] = z[k];
            if (!active[k]) continue;  /* a finished mass keeps its solution */
            zn[k] = z[k] * zo[k] * alpha_o /
                    (alpha * beta_o * (zo[k] - z[k]) + zo[k] * alpha_o * (1.0 + sm[k] * alpha));
            double ak = alpha * zn[k] / z[k];
            cplx *xk = x + (long)k * N, *p_k = pk + (long)k * N;
            for (long j = 0; j < N; ++j) xk[j] += ak * p_k[j];
        }
        for (long j = 0; j < N; ++j) r[j] -= alpha * q[j];
        double rr_new = vnorm2(N, r), beta = rr_new / rr;
        ++iters;
        for (int k = 0; k < nm; ++k) {
            if (active[k]) {
                double bk = beta * (zn[k] / z[k]) * (zn[k] / z[k]);
                cplx *p_k = pk + (long)k * N;
                for (long j = 0; j < N; ++j) p_k[j] = zn[k] * r[j] + bk * p_k[j];
                if (fabs(zn[k]) * sqrt(rr_new) <= tol * bh) active[k] = 0;
            }
            if (zn[k] != z[k]) {
                zo[k] = z[k];
                z[k] = zn[k];
            }
        }
        for (long j = 0; j < N; ++j) p[j] = r[j] + beta * p[j];
        alpha_o = alpha;
        beta_o = beta;
        rr = rr_new;
    }
    /* x_k = y_k / a_k + low-mode part; true residuals with the two-sign operator */
    double bnorm = sqrt(vnorm2(N, b));
    for (int k = 0; k < nm; ++k) {
        cplx *xk = x + (long)k * N;
        for (long j = 0; j < N; ++j) xk[j] /= am[k];
        for (int i = 0; i < nev2; ++i) {
            const cplx *e = xi + (long)i * N;
            double muk = am[k] * mu[i] + masses[k] * masses[k];
            if (muk > 0)
                for (long j = 0; j < N; ++j) xk[j] += (pb[i] / muk) * e[j];
        }
        ddag_d(&a, rho, masses[k], xk, q, t);
        for (long j = 0; j < N; ++j) q[j] = b[j] - q[j];
        true_res[k] = sqrt(vnorm2(N, q)) / bnorm;
    }
    free(r);
    free(p);
    free(q);
    free(t);
    free(pk);
    free(am);
    free(sm);
    free(z);
    free(zo);
    free(zn);
    free(active);
    free(pb);
    return iters;
}

/* ------------------------------------------------------------------ */
/* gauge-covariant network layer (the learned preconditioner)           */
/* ------------------------------------------------------------------ */
/* The paper has no counterpart; the layer is defined from the parallel
 * transporters of Eq. (2) without spin projectors:
 *   y_c(n) = sum_{c'} sum_{p} W[p][c][c'] (U_p x_{c'})(n),
 * p = 0: identity; p = 1+2mu: U_mu(n) x(n+mu); p = 2+2mu: U_mu(n-mu)^dag x(n-mu)
 * (boundary phases applied), W[p][c][c'] a complex 4x4 spin matrix acting on
 * the spin index.  Fields are [channel][V][4][3]. */
static void transport(const int *d, const double *bc, const cplx *U, const cplx *x, long n, int p,
                      cplx out[12])
{
    if (p == 0) {
        memcpy(out, x + n * 12, sizeof(cplx) * 12);
        return;
    }
    int mu = (p - 1) / 2, fwd = ((p - 1) % 2) == 0;
    double ph;
    long m = neighbour(d, bc, n, mu, fwd ? +1 : -1, &ph);
    const cplx *u = fwd ? U + (n * 4 + mu) * 9 : U + (m * 4 + mu) * 9;
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            cplx v = 0;
            for (int b = 0; b < 3; ++b)
                v += (fwd ? u[3 * a + b] : conj(u[3 * b + a])) * x[m * 12 + 3 * s + b];
            out[3 * s + a] = ph * v;
        }
}

void or_net_layer(const int *d, const double *bc, const cplx *U, int cin, int cout, const cplx *W,
                  const cplx *x, cplx *y)
{
    long V = volume(d);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < V; ++n) {
        for (int co = 0; co < cout; ++co) {
            cplx acc[12] = {0};
            for (int p = 0; p < 9; ++p)
                for (int ci = 0; ci < cin; ++ci) {
                    cplx t[12];
                    transport(d, bc, U, x + (long)ci * V * 12, n, p, t);
                    const cplx *w = W + (((long)p * cout + co) * cin + ci) * 16;
                    for (int s = 0; s < 4; ++s)
                        for (int a = 0; a < 3; ++a) {
                            cplx v = 0;
                            for (int s2 = 0; s2 < 4; ++s2) v += w[4 * s + s2] * t[3 * s2 + a];
                            acc[3 * s + a] += v;
                        }
                }
            memcpy(y + ((long)co * V + n) * 12, acc, sizeof(acc));
        }
    }
}

/* Backward pass of or_net_layer for a real loss L.  gy = dL/dRe(y) + i dL/dIm(y)
 * [cout][V][12]; returns gx (same convention, [cin][V][12]) and gW [9][cout][cin][16]
 * with gW = sum_n gy(n) (U_p x(n))^dagger over colour, i.e. dL/dRe W + i dL/dIm W. */
void or_net_layer_grad(const int *d, const double *bc, const cplx *U, int cin, int cout,
                       const cplx *W, const cplx *x, const cplx *gy, cplx *gx, cplx *gW)
{
    long V = volume(d);
    memset(gW, 0, sizeof(cplx) * 9 * cout * cin * 16);
    /* weight gradient: plain accumulation over sites */
    for (long n = 0; n < V; ++n)
        for (int p = 0; p < 9; ++p)
            for (int ci = 0; ci < cin; ++ci) {
                cplx t[12];
                transport(d, bc, U, x + (long)ci * V * 12, n, p, t);
                for (int co = 0; co < cout; ++co) {
                    const cplx *g = gy + ((long)co * V + n) * 12;
                    cplx *w = gW + (((long)p * cout + co) * cin + ci) * 16;
                    for (int s = 0; s < 4; ++s)
                        for (int s2 = 0; s2 < 4; ++s2) {
                            cplx v = 0;
                            for (int a = 0; a < 3; ++a) v += g[3 * s + a] * conj(t[3 * s2 + a]);
                            w[4 * s + s2] += v;
                        }
                }
            }
    /* input gradient: gx_{c'}(m) = sum over (n, p) reaching m of T_p^dag W^dag gy_c(n),
       computed by scattering from every site n */
    memset(gx, 0, sizeof(cplx) * cin * V * 12);
    for (long n = 0; n < V; ++n)
        for (int p = 0; p < 9; ++p) {
            long m = n;
            double ph = 1.0;
            const cplx *u = NULL;
            int fwd = 0;
            if (p > 0) {
                int mu = (p - 1) / 2;
                fwd = ((p - 1) % 2) == 0;
                m = neighbour(d, bc, n, mu, fwd ? +1 : -1, &ph);
                u = fwd ? U + (n * 4 + mu) * 9 : U + (m * 4 + mu) * 9;
            }
            for (int ci = 0; ci < cin; ++ci)
                for (int co = 0; co < cout; ++co) {
                    const cplx *g = gy + ((long)co * V + n) * 12;
                    const cplx *w = W + (((long)p * cout + co) * cin + ci) * 16;
                    cplx h[12]; /* W^dag gy */
                    for (int s2 = 0; s2 < 4; ++s2)
                        for (int a = 0; a < 3; ++a) {
                            cplx v = 0;
                            for (int s = 0; s < 4; ++s) v += conj(w[4 * s + s2]) * g[3 * s + a];
                            h[3 * s2 + a] = v;
                        }
                    cplx *o = gx + ((long)ci * V + m) * 12;
                    for (int s = 0; s < 4; ++s)
                        for (int b = 0; b < 3; ++b) {
                            cplx v = 0;
                            if (p == 0)
                                v = h[3 * s + b];
                            else
                                for (int a = 0; a < 3; ++a) /* (link)^dag h: link[a][b] conj */
                                    v += conj(fwd ? u[3 * a + b] : conj(u[3 * b + a])) * h[3 * s + a];
                            o[3 * s + b] += ph * v;
                        }
                }
        }
}
