/*
 * FP64 CPU oracle for the non-degenerate twisted-mass shifted solver
 * (arXiv:1805.09584).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the bench's CPU-baseline leg call it; the GPU library never does, and
 * the two share no code.
 *
 * Everything here is written plainly from the paper's definitions, in double
 * precision, with no spin projection, no link compression, no even-odd
 * shortcut inside the stencil and no fused loops:
 *
 *   D_ND  = (D_W (x) I_2) + i mu_bar (Gamma_5 (x) tau_3) - eps_bar (I (x) tau_1)
 *                                                     Sec. 2, Eq. "non-degenerate"
 *   D_W psi(x) = (m+4) psi(x) - 1/2 sum_mu (1-gamma_mu) U_mu(x) psi(x+mu)
 *                             - 1/2 sum_mu (1+gamma_mu) U_mu(x-mu)^+ psi(x-mu)
 *                                                     Sec. 2, Eq. "Wilson", c_sw = 0
 *   even-odd Schur complement on odd sites            Sec. 2 (even-odd reduction)
 *       Mhat = D_oo - D_oe D_ee^-1 D_eo
 *   hermitian Qhat = (Gamma_5 (x) tau_1) Mhat, Qhat^2 = Mhat^+ Mhat
 *                                                     Sec. 2, Eq. "g5tau1-hermiticity"
 *   multi-shift CG for (Qhat^2 + sigma_i) x_i = b     Sec. 1, Eq. "shifted_linear";
 *                                                     Sec. 4.2.2 (MMS-CG)
 *
 * Normalisation.  `paper_norm = 1` uses the paper's form with m + 4 = 1/(2 kappa).
 * `paper_norm = 0` (the default of the library) is the hopping-parameter form,
 * i.e. 2 kappa times the paper's operator:
 *     D = 1 - kappa H + 2 i kappa mu_bar gamma_5 tau_3 - 2 kappa eps_bar tau_1.
 *
 * Gamma matrices: chiral basis, gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 =
 * diag(1,1,-1,-1) (Sec. 2).  gamma_0 = [[0,-1],[-1,0]],
 * gamma_k = [[0,-i sigma_k],[i sigma_k,0]] in 2x2 blocks.
 *
 * Boundary: periodic in space; with `apbc` set, every hop that crosses the
 * time boundary (t = T-1 <-> 0) carries a factor -1.
 *
 * Layouts (complex numbers as interleaved re,im doubles):
 *   links  : [4][T][X][Y][Z][3][3]
 *   full   : [V][2 flavor][4 spin][3 color]
 *   odd    : [V/2][2][4][3], odd half-index = lex >> 1
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int dims[4];        /* T, X, Y, Z */
    double kappa;
    double mu_bar;
    double eps_bar;
    int apbc;           /* antiperiodic in time */
    int paper_norm;     /* 1: paper's form, 0: hopping form */
} or_action;

#define NSC 12          /* spin x color per flavor */
#define NSITE 24        /* complex numbers per site (2 flavors) */

/* ------------------------------------------------------------------ gammas */
static cplx GAMMA[4][4][4];
static cplx GAMMA5[4][4];
static int gamma_ready = 0;

static void mat4_mul(cplx a[4][4], cplx b[4][4], cplx c[4][4]) {
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
            c[i][j] = s;
        }
}

static void init_gamma(void) {
    if (gamma_ready) return;
    memset(GAMMA, 0, sizeof GAMMA);
    /* gamma_0 */
    GAMMA[0][0][2] = -1; GAMMA[0][1][3] = -1; GAMMA[0][2][0] = -1; GAMMA[0][3][1] = -1;
    /* Pauli matrices */
    cplx sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                GAMMA[k + 1][a][2 + b] = -I * sig[k][a][b];
                GAMMA[k + 1][2 + a][b] = I * sig[k][a][b];
            }
    cplx t1[4][4], t2[4][4];
    mat4_mul(GAMMA[0], GAMMA[1], t1);
    mat4_mul(t1, GAMMA[2], t2);
    mat4_mul(t2, GAMMA[3], GAMMA5);
    gamma_ready = 1;
}

/* Export the matrices so the tests can check the Clifford algebra. */
void or_gamma(int mu, double *out /* [4][4] complex */) {
    init_gamma();
    cplx (*g)[4] = (mu == 5) ? GAMMA5 : GAMMA[mu];
    memcpy(out, g, sizeof(cplx) * 16);
}

/* ------------------------------------------------------------------ lattice */
static long volume(const or_action *a) {
    return (long)a->dims[0] * a->dims[1] * a->dims[2] * a->dims[3];
}

static void coords(const or_action *a, long lex, int c[4]) {
    c[3] = lex % a->dims[3]; lex /= a->dims[3];
    c[2] = lex % a->dims[2]; lex /= a->dims[2];
    c[1] = lex % a->dims[1]; lex /= a->dims[1];
    c[0] = (int)lex;
}

static long lexi(const or_action *a, const int c[4]) {
    return ((long)(c[0] * a->dims[1] + c[1]) * a->dims[2] + c[2]) * a->dims[3] + c[3];
}

static int parity(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* Neighbour of x in direction mu (dir = +1 or -1); *sign = -1 when the hop
 * crosses the time boundary and the time boundary is antiperiodic. */
static long neighbour(const or_action *a, long x, int mu, int dir, double *sign) {
    int c[4];
    coords(a, x, c);
    int n = a->dims[mu];
    int v = c[mu] + dir;
    *sign = 1.0;
    if (v < 0 || v >= n) {
        v = (v + n) % n;
        if (mu == 0 && a->apbc) *sign = -1.0;
    }
    c[mu] = v;
    return lexi(a, c);
}

static const cplx *link(const or_action *a, const double *links, int mu, long x) {
    return (const cplx *)links + ((long)mu * volume(a) + x) * 9;
}

/* -------------------------------------------------------- operator pieces */
static double hop_coef(const or_action *a) { return a->paper_norm ? 0.5 : a->kappa; }

/* Site-diagonal part of D_ND as an 8x8 matrix on (flavor, spin), color
 * identity: d0 + i m (gamma_5 (x) tau_3) - e (I (x) tau_1).  Index f*4+s. */
static void diag_block(const or_action *a, cplx B[8][8]) {
    init_gamma();
    double d0, m, e;
    if (a->paper_norm) {
        d0 = 1.0 / (2.0 * a->kappa);
        m = a->mu_bar;
        e = a->eps_bar;
    } else {
        d0 = 1.0;
        m = 2.0 * a->kappa * a->mu_bar;
        e = 2.0 * a->kappa * a->eps_bar;
    }
    const double tau3[2][2] = {{1, 0}, {0, -1}};
    const double tau1[2][2] = {{0, 1}, {1, 0}};
    for (int f = 0; f < 2; f++)
        for (int s = 0; s < 4; s++)
            for (int g = 0; g < 2; g++)
                for (int t = 0; t < 4; t++) {
                    cplx v = 0;
                    if (f == g && s == t) v += d0;
                    v += I * m * GAMMA5[s][t] * tau3[f][g];
                    if (s == t) v -= e * tau1[f][g];
                    B[f * 4 + s][g * 4 + t] = v;
                }
}

/* Inverse of an n x n complex matrix by Gauss-Jordan with partial pivoting. */
static int invert(int n, cplx *A, cplx *Ainv) {
    cplx *M = malloc(sizeof(cplx) * n * 2 * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++)
            M[i * 2 * n + j] = (j < n) ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (cabs(M[r * 2 * n + col]) > cabs(M[piv * 2 * n + col])) piv = r;
        if (cabs(M[piv * 2 * n + col]) == 0.0) { free(M); return -1; }
        if (piv != col)
            for (int j = 0; j < 2 * n; j++) {
                cplx t = M[col * 2 * n + j];
                M[col * 2 * n + j] = M[piv * 2 * n + j];
                M[piv * 2 * n + j] = t;
            }
        cplx p = M[col * 2 * n + col];
        for (int j = 0; j < 2 * n; j++) M[col * 2 * n + j] /= p;
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            cplx f = M[r * 2 * n + col];
            if (f == 0) continue;
            for (int j = 0; j < 2 * n; j++) M[r * 2 * n + j] -= f * M[col * 2 * n + j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Ainv[i * n + j] = M[i * 2 * n + n + j];
    free(M);
    return 0;
}

/* The hop block D(y, y + dir*mu) = coef * (P (x) W): P is a 4x4 spin matrix,
 * W a 3x3 color matrix.  Forward (dir=+1): P = 1 - gamma_mu, W = U_mu(y);
 * backward (dir=-1): P = 1 + gamma_mu, W = U_mu(y-mu)^+. */
static long hop_block(const or_action *a, const double *links, long y, int mu, int dir,
                      cplx *coef, cplx P[4][4], cplx W[3][3]) {
    init_gamma();
    double sign;
    long z = neighbour(a, y, mu, dir, &sign);
    *coef = -hop_coef(a) * sign;
    for (int s = 0; s < 4; s++)
        for (int t = 0; t < 4; t++)
            P[s][t] = (s == t ? 1.0 : 0.0) - dir * GAMMA[mu][s][t];
    if (dir > 0) {
        const cplx *u = link(a, links, mu, y);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) W[i][j] = u[i * 3 + j];
    } else {
        const cplx *u = link(a, links, mu, z);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) W[i][j] = conj(u[j * 3 + i]);
    }
    return z;
}

/* out_f += coef * (P (x) W) in_f for both flavors of one site. */
static void kron_apply(cplx coef, cplx P[4][4], cplx W[3][3], const cplx *in, cplx *out) {
    for (int f = 0; f < 2; f++)
        for (int s = 0; s < 4; s++)
            for (int c = 0; c < 3; c++) {
                cplx acc = 0;
                for (int t = 0; t < 4; t++)
                    for (int d = 0; d < 3; d++)
                        acc += P[s][t] * W[c][d] * in[f * NSC + t * 3 + d];
                out[f * NSC + s * 3 + c] += coef * acc;
            }
}

/* Full-lattice D_ND (dagger = 0) or its adjoint D_ND^+ (dagger = 1).
 * The adjoint is taken block by block: D^+(x, y) = D(y, x)^+. */
void or_dnd(const or_action *a, const double *links, const double *in_, double *out_, int dagger) {
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    long V = volume(a);
    cplx B[8][8];
    diag_block(a, B);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        cplx *o = out + x * NSITE;
        const cplx *ix = in + x * NSITE;
        /* diagonal */
        for (int f = 0; f < 2; f++)
            for (int s = 0; s < 4; s++)
                for (int c = 0; c < 3; c++) {
                    cplx acc = 0;
                    for (int g = 0; g < 2; g++)
                        for (int t = 0; t < 4; t++) {
                            cplx b = dagger ? conj(B[g * 4 + t][f * 4 + s]) : B[f * 4 + s][g * 4 + t];
                            acc += b * ix[g * NSC + t * 3 + c];
                        }
                    o[f * NSC + s * 3 + c] = acc;
                }
        /* hops */
        for (int mu = 0; mu < 4; mu++)
            for (int dir = -1; dir <= 1; dir += 2) {
                cplx coef, P[4][4], W[3][3];
                if (!dagger) {
                    long y = hop_block(a, links, x, mu, dir, &coef, P, W);
                    kron_apply(coef, P, W, in + y * NSITE, o);
                } else {
                    /* D^+(x, y) with y = x + dir*mu equals D(y, x)^+, and
                     * D(y, x) is the hop from y in direction -dir. */
                    double sign;
                    long y = neighbour(a, x, mu, dir, &sign);
                    cplx c2, P2[4][4], W2[3][3];
                    hop_block(a, links, y, mu, -dir, &c2, P2, W2);
                    for (int s = 0; s < 4; s++)
                        for (int t = 0; t < 4; t++) P[s][t] = conj(P2[t][s]);
                    for (int i = 0; i < 3; i++)
                        for (int j = 0; j < 3; j++) W[i][j] = conj(W2[j][i]);
                    coef = conj(c2);
                    kron_apply(coef, P, W, in + y * NSITE, o);
                }
            }
    }
}

/* ------------------------------------------------------- even-odd Schur */
static void embed(const or_action *a, const cplx *half, int par, cplx *full) {
    long V = volume(a);
    memset(full, 0, sizeof(cplx) * V * NSITE);
    for (long x = 0; x < V; x++) {
        int c[4];
        coords(a, x, c);
        if (parity(c) == par) memcpy(full + x * NSITE, half + (x >> 1) * NSITE, sizeof(cplx) * NSITE);
    }
}

static void restrict_par(const or_action *a, const cplx *full, int par, cplx *half) {
    long V = volume(a);
    for (long x = 0; x < V; x++) {
        int c[4];
        coords(a, x, c);
        if (parity(c) == par) memcpy(half + (x >> 1) * NSITE, full + x * NSITE, sizeof(cplx) * NSITE);
    }
}

/* Mhat psi_o = D_oo psi_o - D_oe D_ee^-1 D_eo psi_o  (dagger = 0), or the
 * same Schur complement built from D^+ (dagger = 1), which is Mhat^+ because
 * (D^+)_oo = (D_oo)^+, (D^+)_oe = (D_eo)^+, (D^+)_ee^-1 = (D_ee^-1)^+. */
void or_schur(const or_action *a, const double *links, const double *in_, double *out_, int dagger) {
    long V = volume(a), Vh = V / 2;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    cplx *f1 = malloc(sizeof(cplx) * V * NSITE);
    cplx *f2 = malloc(sizeof(cplx) * V * NSITE);
    cplx *he = malloc(sizeof(cplx) * Vh * NSITE);
    cplx *he2 = malloc(sizeof(cplx) * Vh * NSITE);
    cplx *ho = malloc(sizeof(cplx) * Vh * NSITE);

    embed(a, in, 1, f1);
    or_dnd(a, links, (double *)f1, (double *)f2, dagger);
    restrict_par(a, f2, 1, out);  /* D_oo psi */
    restrict_par(a, f2, 0, he);   /* D_eo psi */

    /* D_ee^-1: invert the site block (same on every site, no clover). */
    cplx B[8][8], Bd[8][8], Binv[8][8];
    diag_block(a, B);
    for (int i = 0; i < 8; i++)
        for (int j = 0; j < 8; j++) Bd[i][j] = dagger ? conj(B[j][i]) : B[i][j];
    invert(8, &Bd[0][0], &Binv[0][0]);
    for (long h = 0; h < Vh; h++)
        for (int f = 0; f < 2; f++)
            for (int s = 0; s < 4; s++)
                for (int c = 0; c < 3; c++) {
                    cplx acc = 0;
                    for (int g = 0; g < 2; g++)
                        for (int t = 0; t < 4; t++)
                            acc += Binv[f * 4 + s][g * 4 + t] * he[h * NSITE + g * NSC + t * 3 + c];
                    he2[h * NSITE + f * NSC + s * 3 + c] = acc;
                }

    embed(a, he2, 0, f1);
    or_dnd(a, links, (double *)f1, (double *)f2, dagger);
    restrict_par(a, f2, 1, ho);   /* D_oe D_ee^-1 D_eo psi */
    for (long i = 0; i < Vh * NSITE; i++) out[i] -= ho[i];

    free(f1); free(f2); free(he); free(he2); free(ho);
}

/* Qhat psi = (gamma_5 (x) tau_1) Mhat psi. */
void or_qhat(const or_action *a, const double *links, const double *in_, double *out_) {
    long Vh = volume(a) / 2;
    cplx *t = malloc(sizeof(cplx) * Vh * NSITE);
    or_schur(a, links, in_, (double *)t, 0);
    init_gamma();
    cplx *out = (cplx *)out_;
    for (long h = 0; h < Vh; h++)
        for (int f = 0; f < 2; f++)
            for (int s = 0; s < 4; s++)
                for (int c = 0; c < 3; c++) {
                    cplx acc = 0;
                    for (int t2 = 0; t2 < 4; t2++) acc += GAMMA5[s][t2] * t[h * NSITE + (1 - f) * NSC + t2 * 3 + c];
                    out[h * NSITE + f * NSC + s * 3 + c] = acc;
                }
    free(t);
}

/* (Qhat^2 + sigma) psi = Mhat^+ Mhat psi + sigma psi. */
void or_qhat2(const or_action *a, const double *links, const double *in_, double *out_, double sigma) {
    long n = volume(a) / 2 * NSITE;
    cplx *t = malloc(sizeof(cplx) * n);
    or_schur(a, links, in_, (double *)t, 0);
    or_schur(a, links, (double *)t, out_, 1);
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    for (long i = 0; i < n; i++) out[i] += sigma * in[i];
    free(t);
}

/* ----------------------------------------------------------- vector algebra */
static double re_dot(long n, const cplx *u, const cplx *v) {
    double s = 0;
    for (long i = 0; i < n; i++) s += creal(conj(u[i]) * v[i]);
    return s;
}

/* Plain CG on (Qhat^2 + sigma) x = b from x = 0.  Stops when
 * |r| <= rho |b| (recursively updated residual) or after maxiter.
 * Returns the iteration count (negative if not converged). */
int or_cg(const or_action *a, const double *links, const double *b_, double sigma,
          double rho, int maxiter, double *x_) {
    long n = volume(a) / 2 * NSITE;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n), *w = malloc(sizeof(cplx) * n);
    for (long i = 0; i < n; i++) { x[i] = 0; r[i] = b[i]; p[i] = b[i]; }
    double bb = re_dot(n, b, b), rr = bb;
    int k;
    for (k = 0; k < maxiter; k++) {
        if (rr <= rho * rho * bb) break;
        or_qhat2(a, links, (double *)p, (double *)w, sigma);
        double alpha = rr / re_dot(n, p, w);
        for (long i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * w[i]; }
        double rr_new = re_dot(n, r, r);
        double beta = rr_new / rr;
        rr = rr_new;
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
    }
    free(r); free(p); free(w);
    return (rr <= rho * rho * bb) ? k : -k;
}

/* Multi-mass-shift CG (Jegerlehner's recursion; Sec. 1 and Sec. 4.2.2):
 * one Krylov space, generated by the base system sigma_0, serves every shift.
 *
 *   shifts sigma[0..nshift-1], strictly descending;  the first `nsolve` must
 *   converge, base sigma_0 = sigma[nsolve-1]; shifts after it are "guess
 *   shifts" (Sec. 4.2.2): iterated along, never required to converge.
 *
 *   init: x_i = 0, r = p = p_i = b, zeta_i = zeta_i^old = 1, alpha^old = 1, beta^old = 0
 *   loop: w = (Qhat^2 + sigma_0) p;  alpha = (r,r)/(p,w)
 *         zeta_i^new = zeta_i zeta_i^old alpha^old /
 *               (alpha beta^old (zeta_i^old - zeta_i) + zeta_i^old alpha^old (1 + alpha D_i)),
 *               D_i = sigma_i - sigma_0
 *         alpha_i = alpha zeta_i^new / zeta_i;   x_i += alpha_i p_i
 *         r -= alpha w;  beta = (r,r)_new/(r,r)
 *         beta_i = beta (zeta_i^new/zeta_i)^2;   p_i = zeta_i^new r + beta_i p_i
 *         p = r + beta p
 *   shift i is frozen once |zeta_i| |r| <= rho |b| (its residual is zeta_i r).
 *
 * Outputs: x [nshift][n], conv_iter[nshift] (iteration after which shift i
 * froze, -1 if never), zeta[nshift] final.  Returns the iteration count
 * (negative if the base did not converge within maxiter). */
int or_mms_cg(const or_action *a, const double *links, const double *b_, int nshift, int nsolve,
              const double *sigma, double rho, int maxiter, double *x_, int *conv_iter, double *zeta_out) {
    long n = volume(a) / 2 * NSITE;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n), *w = malloc(sizeof(cplx) * n);
    cplx *ps = malloc(sizeof(cplx) * n * nshift);
    double *zeta = malloc(sizeof(double) * nshift), *zeta_old = malloc(sizeof(double) * nshift);
    int *active = malloc(sizeof(int) * nshift);
    double *zeta_new = malloc(sizeof(double) * nshift), *alpha_s = malloc(sizeof(double) * nshift);
    double sigma0 = sigma[nsolve - 1];
    for (long i = 0; i < n; i++) { r[i] = b[i]; p[i] = b[i]; }
    for (int s = 0; s < nshift; s++) {
        for (long i = 0; i < n; i++) { x[s * n + i] = 0; ps[s * n + i] = b[i]; }
        zeta[s] = zeta_old[s] = 1.0;
        active[s] = 1;
        conv_iter[s] = -1;
    }
    double bb = re_dot(n, b, b), rr = bb;
    double alpha_old = 1.0, beta_old = 0.0;
    int k = 0;
    while (k < maxiter && active[nsolve - 1]) {
        or_qhat2(a, links, (double *)p, (double *)w, sigma0);
        double alpha = rr / re_dot(n, p, w);
        for (int s = 0; s < nshift; s++) {
            if (!active[s]) continue;
            double d = sigma[s] - sigma0;
            zeta_new[s] = zeta[s] * zeta_old[s] * alpha_old /
                          (alpha * beta_old * (zeta_old[s] - zeta[s]) + zeta_old[s] * alpha_old * (1.0 + alpha * d));
            alpha_s[s] = alpha * zeta_new[s] / zeta[s];
            for (long i = 0; i < n; i++) x[s * n + i] += alpha_s[s] * ps[s * n + i];
        }
        for (long i = 0; i < n; i++) r[i] -= alpha * w[i];
        double rr_new = re_dot(n, r, r);
        double beta = rr_new / rr;
        k++;
        for (int s = 0; s < nshift; s++) {
            if (!active[s]) continue;
            double beta_s = beta * (zeta_new[s] / zeta[s]) * (zeta_new[s] / zeta[s]);
            for (long i = 0; i < n; i++) ps[s * n + i] = zeta_new[s] * r[i] + beta_s * ps[s * n + i];
            zeta_old[s] = zeta[s];
            zeta[s] = zeta_new[s];
            if (s < nsolve && fabs(zeta[s]) * sqrt(rr_new) <= rho * sqrt(bb)) {
                active[s] = 0;
                conv_iter[s] = k;
            }
        }
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        rr = rr_new;
        alpha_old = alpha;
        beta_old = beta;
    }
    for (int s = 0; s < nshift; s++) zeta_out[s] = zeta[s];
    int ok = !active[nsolve - 1];
    free(r); free(p); free(w); free(ps); free(zeta); free(zeta_old); free(active);
    free(zeta_new); free(alpha_s);
    return ok ? k : -k;
}
