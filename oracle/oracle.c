/*
 * oracle.c -- plain FP64 CPU oracle for the cell-list force evaluation of
 * Dobson, Fox & Saracino, "Cell List Algorithms for Nonequilibrium Molecular
 * Dynamics" (arXiv:1412.3784).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path and must never be called from the product path.
 *
 * Built with -O2 -ffp-contract=off: every floating-point operation below is a
 * single IEEE round-to-nearest operation in the order written; there is no
 * fused multiply-add.  Slow and obvious on purpose.
 *
 * What it computes, with the passage each part follows:
 *   - lattice evolution L_t = exp(tau A) L0, tau = t mod T        (Sec. 2.1, 2.2, Eq. kr)
 *     exp by the symmetric eigen-decomposition (cyclic Jacobi) when A is
 *     symmetric, else by [13/13] Pade scaling-and-squaring (Higham 2005)
 *   - box heights h_i = V / |v_j x v_k|                            (Sec. 4.1, Fig. bh)
 *   - QR of the box, R upper triangular with positive diagonal   (Sec. 4.2, Eq. R)
 *   - fractional wrap s = frac(L^-1 q), canonical q' = L s         (Sec. 2, unit cell Omega)
 *   - brute-force all-pairs sum over lattice images within rc      (Sec. 3, naive O(N^2))
 *   - dynamic size cell list, c_i = floor(h_i / d_cut), 27 cells   (Sec. 4.1)
 *   - dynamic offset cell list: brick rearrangement and the
 *     expanded boundary neighbourhoods                            (Sec. 4.2, Sec. 5.2)
 *   - LJ / WCA force, energy and virial                           (Sec. 5: force after a distance check)
 *
 * Readings of the paper used here (the paper is silent or garbled):
 *   - the remap is L <- L M^-1 at each period, so L(t) = exp(A (t mod T)) L0;
 *   - the x-rearrangement of the brick wraps modulo r11 (the printed r22 is a typo);
 *   - the cut-off test is strict, r^2 < rc^2;
 *   - cell counts use a relative safety margin of 1e-12:
 *       c_i = floor((1 - 1e-12) h_i / rc),  l_i = floor((1 - 1e-12) r_ii / rc),
 *     and stencil intervals use rc_e = rc (1 + 1e-12), so that rounding of
 *     positions can never drop a pair.
 *
 * Canonical pair definition (identical for brute force and both cell lists):
 *   d(i,j,n)_a = (q'_j,a - q'_i,a) + ((n1 L_a0 + n2 L_a1) + n3 L_a2)
 *   r2 = (d0 d0 + d1 d1) + d2 d2 ;  pair iff r2 < rc*rc and (i,j,n) != (i,i,0)
 *   unordered: (i,j,n) ~ (j,i,-n); reported with i < j, or i == j and n > 0
 *   lexicographically.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MARGIN 1e-12

/* ------------------------------------------------------------------------ */
/* 3x3 matrices, row-major                                                    */
/* ------------------------------------------------------------------------ */

static void m3_mul(const double *a, const double *b, double *c)
{
    double t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            t[3 * i + j] = (a[3 * i + 0] * b[0 + j] + a[3 * i + 1] * b[3 + j]) + a[3 * i + 2] * b[6 + j];
    memcpy(c, t, sizeof t);
}

static double m3_det(const double *a)
{
    return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
           a[2] * (a[3] * a[7] - a[4] * a[6]);
}

/* Inverse by the adjugate divided by the determinant. */
static void m3_inv(const double *a, double *inv, double *det_out)
{
    double det = m3_det(a);
    double c[9];
    c[0] = a[4] * a[8] - a[5] * a[7];
    c[1] = a[2] * a[7] - a[1] * a[8];
    c[2] = a[1] * a[5] - a[2] * a[4];
    c[3] = a[5] * a[6] - a[3] * a[8];
    c[4] = a[0] * a[8] - a[2] * a[6];
    c[5] = a[2] * a[3] - a[0] * a[5];
    c[6] = a[3] * a[7] - a[4] * a[6];
    c[7] = a[1] * a[6] - a[0] * a[7];
    c[8] = a[0] * a[4] - a[1] * a[3];
    for (int k = 0; k < 9; k++) inv[k] = c[k] / det;
    if (det_out) *det_out = det;
}

static double m3_norm1(const double *a)
{
    double best = 0.0;
    for (int j = 0; j < 3; j++) {
        double s = fabs(a[j]) + fabs(a[3 + j]) + fabs(a[6 + j]);
        if (s > best) best = s;
    }
    return best;
}

/* Solve X B = ... : here X = Q^-1 P for 3x3 by Gaussian elimination with
 * partial pivoting on the augmented system Q X = P. */
static void m3_solve(const double *Q, const double *P, double *X)
{
    double a[3][6];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) {
            a[i][j] = Q[3 * i + j];
            a[i][3 + j] = P[3 * i + j];
        }
    }
    for (int col = 0; col < 3; col++) {
        int piv = col;
        for (int r = col + 1; r < 3; r++)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int j = 0; j < 6; j++) {
                double t = a[col][j];
                a[col][j] = a[piv][j];
                a[piv][j] = t;
            }
        for (int r = col + 1; r < 3; r++) {
            double f = a[r][col] / a[col][col];
            for (int j = col; j < 6; j++) a[r][j] = a[r][j] - f * a[col][j];
        }
    }
    for (int j = 0; j < 3; j++) {
        for (int i = 2; i >= 0; i--) {
            double s = a[i][3 + j];
            for (int k = i + 1; k < 3; k++) s = s - a[i][k] * X[3 * k + j];
            X[3 * i + j] = s / a[i][i];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Matrix exponential                                                         */
/* ------------------------------------------------------------------------ */

/* Symmetric case: cyclic Jacobi rotations give A = V diag(mu) V^T, then
 * exp(tau A) = V diag(exp(tau mu)) V^T. */
static void expm_sym(const double *A, double tau, double *E)
{
    double a[9], v[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(a, A, sizeof a);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = fabs(a[1]) + fabs(a[2]) + fabs(a[5]);
        if (off == 0.0) break;
        for (int p = 0; p < 2; p++) {
            for (int q = p + 1; q < 3; q++) {
                double apq = a[3 * p + q];
                if (apq == 0.0) continue;
                double app = a[3 * p + p], aqq = a[3 * q + q];
                double theta = (aqq - app) / (2.0 * apq);
                double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
                /* a <- J^T a J with J the rotation in the (p,q) plane */
                for (int k = 0; k < 3; k++) {
                    double akp = a[3 * k + p], akq = a[3 * k + q];
                    a[3 * k + p] = c * akp - s * akq;
                    a[3 * k + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; k++) {
                    double apk = a[3 * p + k], aqk = a[3 * q + k];
                    a[3 * p + k] = c * apk - s * aqk;
                    a[3 * q + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; k++) {
                    double vkp = v[3 * k + p], vkq = v[3 * k + q];
                    v[3 * k + p] = c * vkp - s * vkq;
                    v[3 * k + q] = s * vkp + c * vkq;
                }
                a[3 * p + q] = 0.0;
                a[3 * q + p] = 0.0;
            }
        }
    }
    double ex[3] = {exp(tau * a[0]), exp(tau * a[4]), exp(tau * a[8])};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            E[3 * i + j] = (v[3 * i + 0] * ex[0] * v[3 * j + 0] + v[3 * i + 1] * ex[1] * v[3 * j + 1]) +
                           v[3 * i + 2] * ex[2] * v[3 * j + 2];
}

/* General case: [13/13] Pade approximant with scaling and squaring
 * (N. J. Higham, SIAM J. Matrix Anal. Appl. 26 (2005) 1179-1193). */
static void expm_pade13(const double *A, double tau, double *E)
{
    static const double b[14] = {64764752532480000.0, 32382376266240000.0, 7771770303897600.0,
                                 1187353796428800.0,  129060195264000.0,   10559470521600.0,
                                 670442572800.0,      33522128640.0,       1323241920.0,
                                 40840800.0,          960960.0,            16380.0,
                                 182.0,               1.0};
    const double theta13 = 5.371920351148152;
    double X[9];
    for (int k = 0; k < 9; k++) X[k] = tau * A[k];
    double nrm = m3_norm1(X);
    int s = 0;
    if (nrm > theta13) s = (int)ceil(log2(nrm / theta13));
    double scale = ldexp(1.0, -s);
    for (int k = 0; k < 9; k++) X[k] *= scale;
    double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    double X2[9], X4[9], X6[9];
    m3_mul(X, X, X2);
    m3_mul(X2, X2, X4);
    m3_mul(X4, X2, X6);
    double U1[9], U[9], V1[9], V[9], T9[9];
    for (int k = 0; k < 9; k++) T9[k] = b[13] * X6[k] + b[11] * X4[k] + b[9] * X2[k];
    m3_mul(X6, T9, U1);
    for (int k = 0; k < 9; k++) U1[k] = U1[k] + b[7] * X6[k] + b[5] * X4[k] + b[3] * X2[k] + b[1] * I[k];
    m3_mul(X, U1, U);
    for (int k = 0; k < 9; k++) T9[k] = b[12] * X6[k] + b[10] * X4[k] + b[8] * X2[k];
    m3_mul(X6, T9, V1);
    for (int k = 0; k < 9; k++) V[k] = V1[k] + b[6] * X6[k] + b[4] * X4[k] + b[2] * X2[k] + b[0] * I[k];
    double P[9], Q[9];
    for (int k = 0; k < 9; k++) {
        P[k] = V[k] + U[k];
        Q[k] = V[k] - U[k];
    }
    double R[9];
    m3_solve(Q, P, R);
    for (int i = 0; i < s; i++) m3_mul(R, R, R);
    memcpy(E, R, sizeof R);
}

int orc_is_symmetric(const double *A)
{
    return A[1] == A[3] && A[2] == A[6] && A[5] == A[7];
}

void orc_expm(const double *A, double tau, double *E)
{
    if (orc_is_symmetric(A))
        expm_sym(A, tau, E);
    else
        expm_pade13(A, tau, E);
}

/* ------------------------------------------------------------------------ */
/* Lattice at time t: out = [L(9), Linv(9), V, h(3), Q(9), R(9)] = 40 doubles */
/* ------------------------------------------------------------------------ */

/* Time within the current remap period: tau in [0, T) (the remap happens at
 * the end of each period), or, centred, tau in [-T/2, T/2) (the remap happens
 * half way, as for the shear flow remapped at half a lattice spacing, Sec. 2.2). */
static double reduce_time(double T, double t, int centered)
{
    if (!(T > 0.0)) return t;
    if (centered) return t - T * floor(t / T + 0.5);
    return t - T * floor(t / T);
}

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm3(const double *a) { return sqrt((a[0] * a[0] + a[1] * a[1]) + a[2] * a[2]); }

/* Columns of L are the lattice vectors; extract column j. */
static void col3(const double *L, int j, double *v)
{
    v[0] = L[j];
    v[1] = L[3 + j];
    v[2] = L[6 + j];
}

void orc_heights(const double *L, double *h)
{
    double v[3][3], c[3];
    for (int j = 0; j < 3; j++) col3(L, j, v[j]);
    double V = fabs(m3_det(L));
    cross3(v[1], v[2], c);
    h[0] = V / norm3(c);
    cross3(v[2], v[0], c);
    h[1] = V / norm3(c);
    cross3(v[0], v[1], c);
    h[2] = V / norm3(c);
}

/* Modified Gram-Schmidt on the columns: L = Q R, r_ii > 0. */
void orc_qr(const double *L, double *Q, double *R)
{
    double v[3][3], q[3][3];
    for (int j = 0; j < 3; j++) col3(L, j, v[j]);
    memset(R, 0, 9 * sizeof(double));
    for (int j = 0; j < 3; j++) {
        double u[3] = {v[j][0], v[j][1], v[j][2]};
        for (int k = 0; k < j; k++) {
            double r = (q[k][0] * u[0] + q[k][1] * u[1]) + q[k][2] * u[2];
            R[3 * k + j] = r;
            for (int a = 0; a < 3; a++) u[a] = u[a] - r * q[k][a];
        }
        double nrm = norm3(u);
        R[3 * j + j] = nrm;
        for (int a = 0; a < 3; a++) q[j][a] = u[a] / nrm;
    }
    for (int a = 0; a < 3; a++)
        for (int j = 0; j < 3; j++) Q[3 * a + j] = q[j][a];
}

void orc_lattice(const double *A, const double *L0, double T, double t, int centered, double *out)
{
    double tau = reduce_time(T, t, centered);
    double E[9];
    orc_expm(A, tau, E);
    double *L = out, *Linv = out + 9, *h = out + 19, *Q = out + 22, *R = out + 31;
    m3_mul(E, L0, L);
    double det;
    m3_inv(L, Linv, &det);
    out[18] = det;
    orc_heights(L, h);
    orc_qr(L, Q, R);
}

/* max_ab |exp(T A) L0 - L0 M|_ab / max_ab |L0_ab| : the KR condition, Eq. kr. */
double orc_kr_residual(const double *A, const double *L0, const int64_t *M, double T)
{
    double E[9], EL[9], LM[9], Mf[9];
    orc_expm(A, T, E);
    m3_mul(E, L0, EL);
    for (int k = 0; k < 9; k++) Mf[k] = (double)M[k];
    m3_mul(L0, Mf, LM);
    double num = 0.0, den = 0.0;
    for (int k = 0; k < 9; k++) {
        if (fabs(EL[k] - LM[k]) > num) num = fabs(EL[k] - LM[k]);
        if (fabs(L0[k]) > den) den = fabs(L0[k]);
    }
    return num / den;
}

/* ------------------------------------------------------------------------ */
/* Wrap into the unit cell and the canonical displacement                     */
/* ------------------------------------------------------------------------ */

void orc_wrap(const double *L, const double *Linv, int64_t n, const double *q, double *s_out, double *qp_out)
{
    for (int64_t i = 0; i < n; i++) {
        const double *x = q + 3 * i;
        double s[3];
        for (int a = 0; a < 3; a++) {
            double v = (Linv[3 * a + 0] * x[0] + Linv[3 * a + 1] * x[1]) + Linv[3 * a + 2] * x[2];
            v = v - floor(v);
            if (v >= 1.0) v = 0.0;
            s[a] = v;
        }
        for (int a = 0; a < 3; a++) {
            s_out[3 * i + a] = s[a];
            qp_out[3 * i + a] = (L[3 * a + 0] * s[0] + L[3 * a + 1] * s[1]) + L[3 * a + 2] * s[2];
        }
    }
}

static inline double canon_r2(const double *qpi, const double *qpj, const double *L, int n1, int n2, int n3,
                              double *d)
{
    double f1 = (double)n1, f2 = (double)n2, f3 = (double)n3;
    for (int a = 0; a < 3; a++) {
        double img = (f1 * L[3 * a + 0] + f2 * L[3 * a + 1]) + f3 * L[3 * a + 2];
        d[a] = (qpj[a] - qpi[a]) + img;
    }
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* ------------------------------------------------------------------------ */
/* Pair accumulation (LJ / WCA)                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    double rc, rc2, eps, sigma, ushift;
    const double *L, *qp;
    int32_t *pairs;   /* 5 ints per pair: i, j, n1, n2, n3 */
    int64_t cap, npairs, ncand;
    double *F;        /* N x 3 in input order, may be NULL */
    double U, W[9];
} acc_t;

static void acc_init(acc_t *ac, const double *L, const double *qp, double rc, double eps, double sigma, int shift,
                     int32_t *pairs, int64_t cap, double *F, int64_t n)
{
    memset(ac, 0, sizeof *ac);
    ac->rc = rc;
    ac->rc2 = rc * rc;
    ac->eps = eps;
    ac->sigma = sigma;
    if (shift) {
        double sr2 = (sigma * sigma) / (rc * rc);
        double sr6 = sr2 * sr2 * sr2;
        ac->ushift = 4.0 * eps * (sr6 * sr6 - sr6);
    }
    ac->L = L;
    ac->qp = qp;
    ac->pairs = pairs;
    ac->cap = cap;
    ac->F = F;
    if (F) memset(F, 0, (size_t)n * 3 * sizeof(double));
}

static int canonical_orientation(int64_t i, int64_t j, int n1, int n2, int n3)
{
    if (i < j) return 1;
    if (i > j) return 0;
    if (n1 != 0) return n1 > 0;
    if (n2 != 0) return n2 > 0;
    return n3 > 0;
}

/* Test one ordered candidate; accumulate it only in canonical orientation so
 * every unordered pair enters the sums once. */
static void acc_candidate(acc_t *ac, int64_t i, int64_t j, int n1, int n2, int n3)
{
    if (i == j && n1 == 0 && n2 == 0 && n3 == 0) return;
    ac->ncand++;
    if (!canonical_orientation(i, j, n1, n2, n3)) return;
    double d[3];
    double r2 = canon_r2(ac->qp + 3 * i, ac->qp + 3 * j, ac->L, n1, n2, n3, d);
    if (!(r2 < ac->rc2)) return;
    if (ac->pairs && ac->npairs < ac->cap) {
        int32_t *p = ac->pairs + 5 * ac->npairs;
        p[0] = (int32_t)i;
        p[1] = (int32_t)j;
        p[2] = n1;
        p[3] = n2;
        p[4] = n3;
    }
    ac->npairs++;
    double r2inv = 1.0 / r2;
    double sr2 = (ac->sigma * ac->sigma) * r2inv;
    double sr6 = sr2 * sr2 * sr2;
    double u = 4.0 * ac->eps * (sr6 * sr6 - sr6) - ac->ushift;
    double fr = 24.0 * ac->eps * r2inv * sr6 * (2.0 * sr6 - 1.0);
    ac->U += u;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) ac->W[3 * a + b] += fr * d[a] * d[b];
    if (ac->F) {
        for (int a = 0; a < 3; a++) {
            ac->F[3 * i + a] -= fr * d[a];
            ac->F[3 * j + a] += fr * d[a];
        }
    }
}

static void acc_finish(const acc_t *ac, double *UW, int64_t *stats)
{
    if (UW) {
        UW[0] = ac->U;
        for (int k = 0; k < 9; k++) UW[1 + k] = ac->W[k];
    }
    if (stats) {
        stats[0] = ac->npairs;
        stats[1] = ac->ncand;
    }
}

/* ------------------------------------------------------------------------ */
/* Brute force: every pair, every lattice image that can lie within rc        */
/* ------------------------------------------------------------------------ */

/* stats[0] = unordered pairs found, stats[1] = ordered candidates tested.
 * Returns the number of pairs (may exceed cap; only cap are written). */
int64_t orc_brute(const double *L, int64_t n, const double *s, const double *qp, double rc, double eps, double sigma,
                  int shift, int32_t *pairs, int64_t cap, double *F, double *UW, int64_t *stats)
{
    double h[3];
    orc_heights(L, h);
    acc_t ac;
    acc_init(&ac, L, qp, rc, eps, sigma, shift, pairs, cap, F, n);
    for (int64_t i = 0; i < n; i++) {
        for (int64_t j = i; j < n; j++) {
            int lo[3], hi[3];
            for (int a = 0; a < 3; a++) {
                double ds = s[3 * j + a] - s[3 * i + a];
                double reach = rc / h[a] + 1e-9;
                lo[a] = (int)ceil(-ds - reach);
                hi[a] = (int)floor(-ds + reach);
            }
            for (int n1 = lo[0]; n1 <= hi[0]; n1++)
                for (int n2 = lo[1]; n2 <= hi[1]; n2++)
                    for (int n3 = lo[2]; n3 <= hi[2]; n3++) acc_candidate(&ac, i, j, n1, n2, n3);
        }
    }
    acc_finish(&ac, UW, stats);
    return ac.npairs;
}

/* ------------------------------------------------------------------------ */
/* Cell lists                                                                 */
/* ------------------------------------------------------------------------ */

static int64_t floordiv(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

/* Cell counts of the dynamic size list: c_i = floor(kfac h_i / rc) with the margin. */
void orc_ds_counts(const double *L, double rc, int kfac, int64_t *c)
{
    double h[3];
    orc_heights(L, h);
    for (int a = 0; a < 3; a++) c[a] = (int64_t)floor((1.0 - ORC_MARGIN) * (double)kfac * h[a] / rc);
}

/* Cell counts of the dynamic offset list: l_i = floor(kfac r_ii / rc). */
void orc_do_counts(const double *R, double rc, int kfac, int64_t *l)
{
    for (int a = 0; a < 3; a++) l[a] = (int64_t)floor((1.0 - ORC_MARGIN) * (double)kfac * R[4 * a] / rc);
}

typedef struct {
    int64_t ncell;
    int64_t *head, *next;
} linked_t;

static int linked_build(linked_t *lk, int64_t ncell, int64_t n, const int64_t *cell_of)
{
    lk->ncell = ncell;
    lk->head = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    lk->next = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!lk->head || !lk->next) return -1;
    for (int64_t c = 0; c < ncell; c++) lk->head[c] = -1;
    /* insert in reverse so each cell lists particles in increasing index */
    for (int64_t i = n - 1; i >= 0; i--) {
        lk->next[i] = lk->head[cell_of[i]];
        lk->head[cell_of[i]] = i;
    }
    return 0;
}

static void linked_free(linked_t *lk)
{
    free(lk->head);
    free(lk->next);
}

/* Dynamic size cell list (Sec. 4.1).  Cells are congruent to the box; a
 * particle goes to cell floor(s_a c_a); the neighbourhood is the 27 (or
 * (2k+1)^3) cells around it, each with the lattice image its wrap implies. */
int64_t orc_cells_ds(const double *L, int64_t n, const double *s, const double *qp, double rc, int kfac, double eps,
                     double sigma, int shift, int32_t *pairs, int64_t cap, double *F, double *UW, int64_t *stats)
{
    int64_t c[3];
    orc_ds_counts(L, rc, kfac, c);
    if (c[0] < 1 || c[1] < 1 || c[2] < 1) return -1;
    int64_t ncell = c[0] * c[1] * c[2];
    int64_t *cell_of = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int64_t idx[3];
        for (int a = 0; a < 3; a++) {
            int64_t k = (int64_t)floor(s[3 * i + a] * (double)c[a]);
            if (k > c[a] - 1) k = c[a] - 1;
            if (k < 0) k = 0;
            idx[a] = k;
        }
        cell_of[i] = idx[0] + c[0] * (idx[1] + c[1] * idx[2]);
    }
    linked_t lk;
    linked_build(&lk, ncell, n, cell_of);
    acc_t ac;
    acc_init(&ac, L, qp, rc, eps, sigma, shift, pairs, cap, F, n);
    int K = kfac;
    for (int64_t iz = 0; iz < c[2]; iz++)
        for (int64_t iy = 0; iy < c[1]; iy++)
            for (int64_t ix = 0; ix < c[0]; ix++) {
                int64_t home = ix + c[0] * (iy + c[1] * iz);
                for (int dz = -K; dz <= K; dz++)
                    for (int dy = -K; dy <= K; dy++)
                        for (int dx = -K; dx <= K; dx++) {
                            int64_t u[3] = {ix + dx, iy + dy, iz + dz}, w[3], img[3];
                            for (int a = 0; a < 3; a++) {
                                img[a] = floordiv(u[a], c[a]);
                                w[a] = u[a] - img[a] * c[a];
                            }
                            int64_t nb = w[0] + c[0] * (w[1] + c[1] * w[2]);
                            for (int64_t i = lk.head[home]; i >= 0; i = lk.next[i])
                                for (int64_t j = lk.head[nb]; j >= 0; j = lk.next[j])
                                    acc_candidate(&ac, i, j, (int)img[0], (int)img[1], (int)img[2]);
                        }
            }
    acc_finish(&ac, UW, stats);
    linked_free(&lk);
    free(cell_of);
    return ac.npairs;
}

/* ------------------------------------------------------------------------ */
/* Dynamic offset cell list (Sec. 4.2)                                        */
/* ------------------------------------------------------------------------ */

/* Rearrange a fractional position into the rectangular brick
 * [0,r11) x [0,r22) x [0,r33) of the rotated lattice R: first z, then y,
 * then x, each time subtracting the lattice vector that undoes the overflow.
 * Returns the brick point b and the integer m with b = R (s - m). */
static void brick_wrap(const double *R, const double *s, double *b, int64_t *m)
{
    double x = (R[0] * s[0] + R[1] * s[1]) + R[2] * s[2];
    double y = R[4] * s[1] + R[5] * s[2];
    double z = R[8] * s[2];
    double m3 = floor(z / R[8]);
    z = z - m3 * R[8];
    y = y - m3 * R[5];
    x = x - m3 * R[2];
    double m2 = floor(y / R[4]);
    y = y - m2 * R[4];
    x = x - m2 * R[1];
    double m1 = floor(x / R[0]);
    x = x - m1 * R[0];
    b[0] = x;
    b[1] = y;
    b[2] = z;
    m[0] = (int64_t)m1;
    m[1] = (int64_t)m2;
    m[2] = (int64_t)m3;
}

/* One neighbour row of the dynamic offset stencil for a home cell row (iy, iz):
 * the x-cells [ix+dxlo, ix+dxhi] of unwrapped row jyu in unwrapped layer jzu. */
typedef struct {
    int64_t jyu, jzu, dxlo, dxhi;
} dorow_t;

/* Tight rule: every layer / row / x-run whose cells intersect the home cell
 * expanded by rc_e.  Returns the number of rows written (at most cap). */
static int do_rows(const double *R, const int64_t *l, double rc, int64_t iy, int64_t iz, dorow_t *rows, int cap)
{
    double w[3] = {R[0] / (double)l[0], R[4] / (double)l[1], R[8] / (double)l[2]};
    double rce = rc * (1.0 + ORC_MARGIN);
    int nr = 0;
    int64_t zlo = (int64_t)floor(((double)iz * w[2] - rce) / w[2]);
    int64_t zhi = (int64_t)ceil(((double)(iz + 1) * w[2] + rce) / w[2]) - 1;
    for (int64_t jzu = zlo; jzu <= zhi; jzu++) {
        int64_t kz = floordiv(jzu, l[2]);
        double yshift = (double)kz * R[5];
        int64_t ylo = (int64_t)floor(((double)iy * w[1] - rce - yshift) / w[1]);
        int64_t yhi = (int64_t)ceil(((double)(iy + 1) * w[1] + rce - yshift) / w[1]) - 1;
        for (int64_t jyu = ylo; jyu <= yhi; jyu++) {
            int64_t ky = floordiv(jyu, l[1]);
            double sx = (double)ky * R[1] + (double)kz * R[2];
            int64_t xlo = (int64_t)floor((-rce - sx) / w[0]);
            int64_t xhi = (int64_t)ceil((w[0] + rce - sx) / w[0]) - 1;
            if (nr < cap) {
                rows[nr].jyu = jyu;
                rows[nr].jzu = jzu;
                rows[nr].dxlo = xlo;
                rows[nr].dxhi = xhi;
            }
            nr++;
        }
    }
    return nr;
}

/* Export the dynamic offset stencil: for every (iy, iz) the rows
 * (iy, iz, jyu, jzu, dxlo, dxhi).  Returns the total row count. */
int64_t orc_do_stencil(const double *R, double rc, int kfac, int64_t *l_out, int64_t *rows_out, int64_t cap)
{
    int64_t l[3];
    orc_do_counts(R, rc, kfac, l);
    for (int a = 0; a < 3; a++) l_out[a] = l[a];
    if (l[0] < 1 || l[1] < 1 || l[2] < 1) return -1;
    int64_t total = 0;
    dorow_t rows[512];
    for (int64_t iz = 0; iz < l[2]; iz++)
        for (int64_t iy = 0; iy < l[1]; iy++) {
            int nr = do_rows(R, l, rc, iy, iz, rows, 512);
            for (int r = 0; r < nr && r < 512; r++) {
                if (total < cap) {
                    int64_t *o = rows_out + 6 * total;
                    o[0] = iy;
                    o[1] = iz;
                    o[2] = rows[r].jyu;
                    o[3] = rows[r].jzu;
                    o[4] = rows[r].dxlo;
                    o[5] = rows[r].dxhi;
                }
                total++;
            }
        }
    return total;
}

/* Number of cells in the neighbourhood of home row (iy, iz) under the paper's
 * fixed expansion rule (Sec. 4.2, four cases): a layer reached across an XY
 * face is 4 x 4 cells, a row reached across an XZ face is 4 cells, every other
 * row is 3 cells.  Needs l2, l3 >= 2. */
int64_t orc_do_fixed_count(const int64_t *l, int64_t iy, int64_t iz)
{
    int64_t total = 0;
    for (int dz = -1; dz <= 1; dz++) {
        int64_t jz = iz + dz;
        if (jz < 0 || jz >= l[2]) {
            total += 16;
            continue;
        }
        for (int dy = -1; dy <= 1; dy++) {
            int64_t jy = iy + dy;
            total += (jy < 0 || jy >= l[1]) ? 4 : 3;
        }
    }
    return total;
}

int64_t orc_cells_do(const double *L, int64_t n, const double *s, const double *qp, double rc, int kfac, double eps,
                     double sigma, int shift, int32_t *pairs, int64_t cap, double *F, double *UW, int64_t *stats)
{
    double Q[9], R[9];
    orc_qr(L, Q, R);
    int64_t l[3];
    orc_do_counts(R, rc, kfac, l);
    if (l[0] < 1 || l[1] < 1 || l[2] < 1) return -1;
    double w[3] = {R[0] / (double)l[0], R[4] / (double)l[1], R[8] / (double)l[2]};
    int64_t ncell = l[0] * l[1] * l[2];
    int64_t *cell_of = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *mimg = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        double b[3];
        brick_wrap(R, s + 3 * i, b, mimg + 3 * i);
        int64_t idx[3];
        for (int a = 0; a < 3; a++) {
            int64_t k = (int64_t)floor(b[a] / w[a]);
            if (k > l[a] - 1) k = l[a] - 1;
            if (k < 0) k = 0;
            idx[a] = k;
        }
        cell_of[i] = idx[0] + l[0] * (idx[1] + l[1] * idx[2]);
    }
    linked_t lk;
    linked_build(&lk, ncell, n, cell_of);
    acc_t ac;
    acc_init(&ac, L, qp, rc, eps, sigma, shift, pairs, cap, F, n);
    dorow_t rows[512];
    for (int64_t iz = 0; iz < l[2]; iz++)
        for (int64_t iy = 0; iy < l[1]; iy++) {
            int nr = do_rows(R, l, rc, iy, iz, rows, 512);
            if (nr > 512) nr = 512;
            for (int64_t ix = 0; ix < l[0]; ix++) {
                int64_t home = ix + l[0] * (iy + l[1] * iz);
                for (int r = 0; r < nr; r++) {
                    int64_t kz = floordiv(rows[r].jzu, l[2]), jz = rows[r].jzu - kz * l[2];
                    int64_t ky = floordiv(rows[r].jyu, l[1]), jy = rows[r].jyu - ky * l[1];
                    for (int64_t dx = rows[r].dxlo; dx <= rows[r].dxhi; dx++) {
                        int64_t jxu = ix + dx;
                        int64_t kx = floordiv(jxu, l[0]), jx = jxu - kx * l[0];
                        int64_t nb = jx + l[0] * (jy + l[1] * jz);
                        /* brick point of j in image k is R (s_j - m_j + k); relative
                         * to i that is the lattice vector n = k - m_j + m_i */
                        for (int64_t i = lk.head[home]; i >= 0; i = lk.next[i])
                            for (int64_t j = lk.head[nb]; j >= 0; j = lk.next[j]) {
                                int64_t n1 = kx - mimg[3 * j + 0] + mimg[3 * i + 0];
                                int64_t n2 = ky - mimg[3 * j + 1] + mimg[3 * i + 1];
                                int64_t n3 = kz - mimg[3 * j + 2] + mimg[3 * i + 2];
                                acc_candidate(&ac, i, j, (int)n1, (int)n2, (int)n3);
                            }
                    }
                }
            }
        }
    acc_finish(&ac, UW, stats);
    linked_free(&lk);
    free(cell_of);
    free(mimg);
    return ac.npairs;
}

/* Total cells over all home neighbourhoods of the tight dynamic offset rule,
 * and of the 27-cell dynamic size rule, for search-volume accounting. */
int64_t orc_do_total_stencil_cells(const double *R, double rc, int kfac)
{
    int64_t l[3];
    orc_do_counts(R, rc, kfac, l);
    if (l[0] < 1 || l[1] < 1 || l[2] < 1) return -1;
    dorow_t rows[512];
    int64_t total = 0;
    for (int64_t iz = 0; iz < l[2]; iz++)
        for (int64_t iy = 0; iy < l[1]; iy++) {
            int nr = do_rows(R, l, rc, iy, iz, rows, 512);
            for (int r = 0; r < nr && r < 512; r++) total += (rows[r].dxhi - rows[r].dxlo + 1) * l[0];
        }
    return total;
}

/* Forces on a sample of particles by brute force over every partner and image:
 * for each sampled i, F_i = sum over (j, n) with r < rc of -fr d, and the number
 * of such (j, n).  Lets full-size runs be checked particle by particle. */
void orc_sample_forces(const double *L, int64_t n, const double *s, const double *qp, double rc, double eps,
                       double sigma, int shift, const int64_t *idx, int64_t nidx, double *F, int64_t *cnt,
                       double *U_half)
{
    (void)shift;
    double h[3];
    orc_heights(L, h);
    double rc2 = rc * rc;
    double ushift = 0.0;
    if (shift) {
        double sr2 = (sigma * sigma) / (rc * rc);
        double sr6 = sr2 * sr2 * sr2;
        ushift = 4.0 * eps * (sr6 * sr6 - sr6);
    }
    for (int64_t t = 0; t < nidx; t++) {
        int64_t i = idx[t];
        double f[3] = {0, 0, 0}, u = 0.0;
        int64_t c = 0;
        for (int64_t j = 0; j < n; j++) {
            int lo[3], hi[3];
            for (int a = 0; a < 3; a++) {
                double ds = s[3 * j + a] - s[3 * i + a];
                double reach = rc / h[a] + 1e-9;
                lo[a] = (int)ceil(-ds - reach);
                hi[a] = (int)floor(-ds + reach);
            }
            for (int n1 = lo[0]; n1 <= hi[0]; n1++)
                for (int n2 = lo[1]; n2 <= hi[1]; n2++)
                    for (int n3 = lo[2]; n3 <= hi[2]; n3++) {
                        if (j == i && n1 == 0 && n2 == 0 && n3 == 0) continue;
                        double d[3];
                        double r2 = canon_r2(qp + 3 * i, qp + 3 * j, L, n1, n2, n3, d);
                        if (!(r2 < rc2)) continue;
                        double r2inv = 1.0 / r2;
                        double sr2 = (sigma * sigma) * r2inv;
                        double sr6 = sr2 * sr2 * sr2;
                        double fr = 24.0 * eps * r2inv * sr6 * (2.0 * sr6 - 1.0);
                        u += 0.5 * (4.0 * eps * (sr6 * sr6 - sr6) - ushift);
                        for (int a = 0; a < 3; a++) f[a] -= fr * d[a];
                        c++;
                    }
        }
        for (int a = 0; a < 3; a++) F[3 * t + a] = f[a];
        cnt[t] = c;
        if (U_half) U_half[t] = u;
    }
}

/* ------------------------------------------------------------------------ */
/* The learned selector's network, FP64 (test oracle of its training kernels) */
/* ------------------------------------------------------------------------ */

/* Layers 12 -> 64 (ReLU) -> 64 (ReLU) -> 4; parameters W1[64][12] b1[64]
 * W2[64][64] b2[64] W3[4][64] b3[4].  Returns L = sum (y - t)^2 / (rows 4) and,
 * if grad is not NULL, dL/dparams by back-propagation.  Y (optional) receives
 * the outputs. */
#define ORC_DI 12
#define ORC_H 64
#define ORC_DO 4
double orc_mlp_loss_grad(const double *p, const double *X, const double *T, int64_t rows, double *grad, double *Y)
{
    const double *W1 = p, *b1 = W1 + ORC_H * ORC_DI, *W2 = b1 + ORC_H, *b2 = W2 + ORC_H * ORC_H, *W3 = b2 + ORC_H,
                 *b3 = W3 + ORC_DO * ORC_H;
    const int np = ORC_H * ORC_DI + ORC_H + ORC_H * ORC_H + ORC_H + ORC_DO * ORC_H + ORC_DO;
    double *gW1 = grad, *gb1 = 0, *gW2 = 0, *gb2 = 0, *gW3 = 0, *gb3 = 0;
    if (grad) {
        memset(grad, 0, sizeof(double) * np);
        gb1 = gW1 + ORC_H * ORC_DI;
        gW2 = gb1 + ORC_H;
        gb2 = gW2 + ORC_H * ORC_H;
        gW3 = gb2 + ORC_H;
        gb3 = gW3 + ORC_DO * ORC_H;
    }
    double loss = 0.0;
    const double scale = 2.0 / (double)(rows * ORC_DO);
    for (int64_t b = 0; b < rows; b++) {
        const double *x = X + b * ORC_DI;
        double h1[ORC_H], h2[ORC_H], y[ORC_DO], d3[ORC_DO], d2[ORC_H], d1[ORC_H];
        for (int h = 0; h < ORC_H; h++) {
            double a = b1[h];
            for (int i = 0; i < ORC_DI; i++) a += W1[h * ORC_DI + i] * x[i];
            h1[h] = a > 0.0 ? a : 0.0;
        }
        for (int h = 0; h < ORC_H; h++) {
            double a = b2[h];
            for (int k = 0; k < ORC_H; k++) a += W2[h * ORC_H + k] * h1[k];
            h2[h] = a > 0.0 ? a : 0.0;
        }
        for (int o = 0; o < ORC_DO; o++) {
            double a = b3[o];
            for (int k = 0; k < ORC_H; k++) a += W3[o * ORC_H + k] * h2[k];
            y[o] = a;
            const double e = a - T[b * ORC_DO + o];
            loss += e * e;
            d3[o] = scale * e;
            if (Y) Y[b * ORC_DO + o] = a;
        }
        if (!grad) continue;
        for (int o = 0; o < ORC_DO; o++) {
            gb3[o] += d3[o];
            for (int k = 0; k < ORC_H; k++) gW3[o * ORC_H + k] += d3[o] * h2[k];
        }
        for (int h = 0; h < ORC_H; h++) {
            double a = 0.0;
            for (int o = 0; o < ORC_DO; o++) a += W3[o * ORC_H + h] * d3[o];
            d2[h] = h2[h] > 0.0 ? a : 0.0;
            gb2[h] += d2[h];
            for (int k = 0; k < ORC_H; k++) gW2[h * ORC_H + k] += d2[h] * h1[k];
        }
        for (int k = 0; k < ORC_H; k++) {
            double a = 0.0;
            for (int h = 0; h < ORC_H; h++) a += W2[h * ORC_H + k] * d2[h];
            d1[k] = h1[k] > 0.0 ? a : 0.0;
            gb1[k] += d1[k];
            for (int i = 0; i < ORC_DI; i++) gW1[k * ORC_DI + i] += d1[k] * x[i];
        }
    }
    return loss / (double)(rows * ORC_DO);
}
