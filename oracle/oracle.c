/*
 * oracle.c -- plain FP64 CPU oracle for the 3x3 Hermitian inverse / determinant path.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load this library.  It shares no
 * source, header, table or helper with the CUDA library: it is written from the
 * paper's definitions, in the order the paper states them, as slow and obvious
 * double-precision loops.  It is single-threaded on purpose.
 *
 * Paper: D. F. G. Coelho, R. J. Cintra, A. C. Frery, V. S. Dimitrov, "Fast Matrix
 * Inversion and Determinant Computation for Polarimetric Synthetic Aperture
 * Radar", arXiv:1807.08084.
 *
 * What each exported function computes, and what pins it (the tests):
 *   oracle_zinv_det        inverse by Gauss-Jordan elimination with partial
 *                          pivoting (the plain definition A X = I; independent of
 *                          the adjugate route of Eq. inv_adjoint), det as the
 *                          product of its pivots (the determinant Eq. det
 *                          expands, evaluated backward-stably: a cofactor
 *                          expansion in FP64 loses u64 cond lmax/lmid, 1e-2 at
 *                          cond 1e7, while elimination keeps u64 cond).  Pinned by exact
 *                          rational arithmetic on a fixed matrix, numpy.linalg on
 *                          random matrices, Z Z^-1 = I, diagonal and block-diagonal
 *                          closed forms (§5), U diag(l) U^H with known l.
 *   oracle_det_expansions  det along each row and column (§3.1: "any of the row or
 *                          column elements weighted by their cofactors").  Pinned
 *                          by the six expansions agreeing and matching numpy.
 *   oracle_inverse_full    full 3x3 inverse by GE or by adj/det (Eq. inv_adjoint),
 *                          so the two derivations can be cross-checked.
 *   oracle_eigvals         eigenvalues by the cyclic Jacobi method for complex
 *                          Hermitian matrices; used for cond_2(Z) = lmax/lmin in
 *                          the tolerances.  Pinned by numpy.linalg.eigvalsh, the
 *                          characteristic-polynomial invariants and constructed
 *                          spectra.
 *   oracle_multilook       Z(p) = sum_k w_k s(p+k) s(p+k)^H over a win x win window
 *                          with clamp-to-edge addressing; boxcar w_k = 1/N gives
 *                          Eq. ZN, (1/N) sum_l S(l) S(l)^H with S a column vector.
 *                          Pinned by brute-force Python loops on tiny images.
 *   oracle_zinv_det_bwd    real packed gradient of L(W, det, log det) w.r.t. the 9
 *                          packed reals of Z.  Pinned by FP64 central finite
 *                          differences through numpy.linalg.
 *   oracle_zinv_det_blockdiag  multifrequency block-diagonal pixels (§5): GE on the
 *                          full 3nb x 3nb matrix.  Pinned by numpy.linalg on the
 *                          full matrix and by the product of the blocks' dets.
 *   oracle_nlm_wishart     nonlocal-means filter of packed Z with the Wishart
 *                          equal-looks distance over a square search window (§1).
 *                          Pinned by constant images, h -> infinity (box mean),
 *                          h -> 0 (identity), d >= 0 with d(i, i) = 0 and
 *                          symmetry, and brute-force numpy.
 *   oracle_stochastic_distance, oracle_nlm_stochastic
 *                          Bhattacharyya, Hellinger, Kullback-Leibler and Renyi distances
 *                          between equal-looks complex Wishart laws (§1's list of
 *                          divergences), in closed form from the Wishart density,
 *                          and the nonlocal-means filter weighted by exp(-d / h).
 *                          Pinned by a Monte Carlo estimate of the defining
 *                          integrals from sampled Wishart matrices, the
 *                          identity S_i^-1 + S_j^-1 = S_i^-1 (S_i + S_j) S_j^-1
 *                          (Bhattacharyya = L x the log-det distance above),
 *                          closed forms for S_j = c S_i and diagonal pairs,
 *                          invariance under a common congruence, symmetry,
 *                          d(i, i) = 0, and brute-force numpy filters.
 *   oracle_wishart_fwd/bwd change statistic q = ln det Z1 + ln det Z2
 *                          - 2 ln det((Z1+Z2)/2) (the log of the likelihood-ratio
 *                          test the paper cites in §1, divided by the number of
 *                          looks), summed over pixels, and its gradient w.r.t. the
 *                          window weights.  Pinned by finite differences, q <= 0,
 *                          q(Z,Z) = 0, Euler homogeneity and date-swap symmetry.
 *
 * Packed Hermitian storage (§2.1: only the upper triangle is stored): nine real
 * planes in the paper's letter order
 *     0:a  1:Re b  2:Im b  3:Re c  4:Im c  5:d  6:Re e  7:Im e  8:f
 * for A = [[a, b, c], [conj b, d, e], [conj c, conj e, f]]; element k of pixel p
 * is at z[k*ld + p].
 *
 * Single-look scattering vectors s = [S_HH, S_HV, S_VV]^T (§1): three complex
 * planes, interleaved (re, im) doubles; component i of pixel (y, x) is at
 * s[2*(i*plane_ld + y*W + x)] (+1 for the imaginary part).
 *
 * ORACLE_MUTANT (compile-time, default 0) plants one deliberate mistake; the test
 * suite builds each mutant and checks that its pins catch it.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#define ORACLE_VERSION 1

typedef double _Complex cplx;

typedef struct {
    cplx m[3][3];
} mat3;

/* ------------------------------------------------------------------------ */
/* Packed storage <-> full matrix (§2.1)                                     */
/* ------------------------------------------------------------------------ */

static mat3 unpack(const double* z, int64_t ld, int64_t p)
{
    double a = z[0 * ld + p];
    cplx b = z[1 * ld + p] + I * z[2 * ld + p];
    cplx c = z[3 * ld + p] + I * z[4 * ld + p];
    double d = z[5 * ld + p];
    cplx e = z[6 * ld + p] + I * z[7 * ld + p];
    double f = z[8 * ld + p];
    mat3 A;
    A.m[0][0] = a;
    A.m[0][1] = b;
    A.m[0][2] = c;
    A.m[1][1] = d;
    A.m[1][2] = e;
    A.m[2][2] = f;
#if ORACLE_MUTANT == 2
    A.m[1][0] = b; /* mutant: lower triangle not conjugated */
#else
    A.m[1][0] = conj(b);
#endif
    A.m[2][0] = conj(c);
    A.m[2][1] = conj(e);
    return A;
}

/* Writes the upper triangle of X into the nine packed planes at pixel p. */
static void pack_upper(const mat3* X, double* out, int64_t ld, int64_t p)
{
#if ORACLE_MUTANT == 3
    /* mutant: packs the lower triangle (conjugated off-diagonals) */
    cplx b = X->m[1][0], c = X->m[2][0], e = X->m[2][1];
#else
    cplx b = X->m[0][1], c = X->m[0][2], e = X->m[1][2];
#endif
    out[0 * ld + p] = creal(X->m[0][0]);
    out[1 * ld + p] = creal(b);
    out[2 * ld + p] = cimag(b);
    out[3 * ld + p] = creal(c);
    out[4 * ld + p] = cimag(c);
    out[5 * ld + p] = creal(X->m[1][1]);
    out[6 * ld + p] = creal(e);
    out[7 * ld + p] = cimag(e);
    out[8 * ld + p] = creal(X->m[2][2]);
}

static void fill_nan(double* out, int64_t ld, int64_t p, int planes)
{
    for (int k = 0; k < planes; ++k) out[k * ld + p] = NAN;
}

/* ------------------------------------------------------------------------ */
/* Cofactors and determinant (§2.1: (i,j) cofactor = (-1)^(i+j) times the   */
/* determinant of A with row i and column j removed; §3.1 Eq. det)          */
/* ------------------------------------------------------------------------ */

/* Determinant of the 2x2 submatrix of A without row i and column j. */
static cplx minor2(const mat3* A, int i, int j)
{
    int r[2], c[2], nr = 0, nc = 0;
    for (int k = 0; k < 3; ++k) {
        if (k != i) r[nr++] = k;
        if (k != j) c[nc++] = k;
    }
    return A->m[r[0]][c[0]] * A->m[r[1]][c[1]] - A->m[r[0]][c[1]] * A->m[r[1]][c[0]];
}

static cplx cofactor(const mat3* A, int i, int j)
{
#if ORACLE_MUTANT == 1
    double sign = (i % 2 == 0) ? 1.0 : -1.0; /* mutant: sign ignores the column */
#else
    double sign = ((i + j) % 2 == 0) ? 1.0 : -1.0;
#endif
    return sign * minor2(A, i, j);
}

/* det A = sum_i A[i][j] * C[i][j] for a fixed column j. */
static cplx det_by_column(const mat3* A, int j)
{
    cplx s = 0;
    for (int i = 0; i < 3; ++i) s += A->m[i][j] * cofactor(A, i, j);
    return s;
}

/* det A = sum_j A[i][j] * C[i][j] for a fixed row i. */
static cplx det_by_row(const mat3* A, int i)
{
    cplx s = 0;
    for (int j = 0; j < 3; ++j) s += A->m[i][j] * cofactor(A, i, j);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Inverse by Gauss-Jordan elimination with partial pivoting on [A | I].     */
/* This is the plain definition (solve A X = I) and uses no cofactor.  The  */
/* same elimination gives det A as the product of the pivots times the sign */
/* of the row permutation.  Both are backward stable: their error is of     */
/* order u * cond(A), whereas a cofactor expansion evaluated in floating    */
/* point loses u * cond(A) * lmax/lmid when two eigenvalues are small.      */
/* Returns 0 on success, -1 if a pivot is exactly zero (singular, det 0).   */
/* ------------------------------------------------------------------------ */

static int ge_inverse_det(const mat3* A, mat3* X, cplx* det)
{
    cplx M[3][6];
    cplx prod = 1.0;
    int swaps = 0;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            M[i][j] = A->m[i][j];
            M[i][3 + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (cabs(M[r][col]) > cabs(M[piv][col])) piv = r;
        if (cabs(M[piv][col]) == 0.0) {
            if (det) *det = 0.0;
            return -1;
        }
        if (piv != col) {
            ++swaps;
            for (int k = 0; k < 6; ++k) {
                cplx t = M[col][k];
                M[col][k] = M[piv][k];
                M[piv][k] = t;
            }
        }
        prod *= M[col][col];
        cplx inv_p = 1.0 / M[col][col];
        for (int k = 0; k < 6; ++k) M[col][k] *= inv_p;
        for (int r = 0; r < 3; ++r) {
            if (r == col) continue;
            cplx factor = M[r][col];
            for (int k = 0; k < 6; ++k) M[r][k] -= factor * M[col][k];
        }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) X->m[i][j] = M[i][3 + j];
#if ORACLE_MUTANT == 11
    if (det) *det = prod; /* mutant: permutation sign ignored */
#else
    if (det) *det = (swaps % 2) ? -prod : prod;
#endif
    return 0;
}

static int ge_inverse(const mat3* A, mat3* X) { return ge_inverse_det(A, X, NULL); }

/* det A by elimination (see ge_inverse_det); 0 for an exactly singular A. */
static cplx det_ge(const mat3* A)
{
    mat3 X;
    cplx d = 0.0;
    ge_inverse_det(A, &X, &d);
    return d;
}

/* Inverse through the adjoint (Eq. inv_adjoint): X[i][j] = C[j][i] / det A. */
static void adj_inverse(const mat3* A, mat3* X)
{
    cplx det = det_by_column(A, 0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) X->m[i][j] = cofactor(A, j, i) / det;
}

/* ------------------------------------------------------------------------ */
/* Eigenvalues of a complex Hermitian 3x3 matrix by the cyclic Jacobi method */
/* (textbook: each step zeroes one off-diagonal pair by a unitary plane      */
/* rotation; sweeps repeat until the off-diagonal mass is negligible).       */
/* lam is returned in ascending order.                                      */
/* ------------------------------------------------------------------------ */

static void matmul3(const mat3* X, const mat3* Y, mat3* out)
{
    mat3 t;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = 0;
            for (int k = 0; k < 3; ++k) s += X->m[i][k] * Y->m[k][j];
            t.m[i][j] = s;
        }
    *out = t;
}

static void adjoint3(const mat3* X, mat3* out)
{
    mat3 t;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) t.m[i][j] = conj(X->m[j][i]);
    *out = t;
}

static void jacobi_eigvals(const mat3* A0, double lam[3])
{
    mat3 A = *A0;
    double fro2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) fro2 += creal(A.m[i][j] * conj(A.m[i][j]));
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off2 = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (i != j) off2 += creal(A.m[i][j] * conj(A.m[i][j]));
        if (off2 <= 1e-34 * fro2 || off2 == 0.0) break;
        for (int p = 0; p < 2; ++p) {
            for (int q = p + 1; q < 3; ++q) {
                double r = cabs(A.m[p][q]);
                if (r == 0.0) continue;
                /* Phase D = diag(1, e^{-i phi}) on the (p,q) plane makes the pair
                   real: [[alpha, r], [r, gamma]].  A real rotation R with
                   t = tan(theta) the smaller root of t^2 + 2 tau t - 1 = 0,
                   tau = (gamma - alpha) / (2 r), then zeroes it. */
                cplx ph = A.m[p][q] / r;
                double alpha = creal(A.m[p][p]), gamma = creal(A.m[q][q]);
                double tau = (gamma - alpha) / (2.0 * r);
#if ORACLE_MUTANT == 9
                double t = 1.0 / (fabs(tau) + sqrt(1.0 + tau * tau)); /* mutant: sign dropped */
#else
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
#endif
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                mat3 J;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) J.m[i][j] = (i == j) ? 1.0 : 0.0;
                J.m[p][p] = c;
                J.m[p][q] = s;
                J.m[q][p] = -s * conj(ph);
                J.m[q][q] = c * conj(ph);
                mat3 Jh, T;
                adjoint3(&J, &Jh);
                matmul3(&A, &J, &T);
                matmul3(&Jh, &T, &A);
                A.m[p][q] = 0.0; /* exact zero in exact arithmetic */
                A.m[q][p] = 0.0;
            }
        }
    }
    double l[3] = {creal(A.m[0][0]), creal(A.m[1][1]), creal(A.m[2][2])};
    /* ascending sort of three values */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2 - i; ++j)
            if (l[j] > l[j + 1]) {
                double tmp = l[j];
                l[j] = l[j + 1];
                l[j + 1] = tmp;
            }
    lam[0] = l[0];
    lam[1] = l[1];
    lam[2] = l[2];
}

/* ------------------------------------------------------------------------ */
/* Exported: per-pixel inverse and determinant                              */
/* ------------------------------------------------------------------------ */

int oracle_version(void) { return ORACLE_VERSION; }

/*
 * z:    [9][ld] packed Hermitian input (§2.1), n pixels.
 * zinv: [9][n] packed upper triangle of Z^-1 by Gauss-Jordan elimination.
 * det:  [n] det Z (real for Hermitian Z, §3.1) from the same elimination: the
 *       value of the cofactor expansion of Eq. det, evaluated backward-stably.
 * det_im (may be NULL): [n] its imaginary part, zero up to rounding.
 * A singular pixel (zero pivot) gets NaN in zinv and det 0.
 */
void oracle_zinv_det(const double* z, int64_t n, int64_t ld, double* zinv, double* det,
                     double* det_im)
{
    for (int64_t p = 0; p < n; ++p) {
        mat3 A = unpack(z, ld, p), X;
        cplx dt = 0.0;
        if (ge_inverse_det(&A, &X, &dt) == 0)
            pack_upper(&X, zinv, n, p);
        else
            fill_nan(zinv, n, p, 9);
        det[p] = creal(dt);
        if (det_im) det_im[p] = cimag(dt);
    }
}

/*
 * out: [12][n]: (re, im) of det expanded along row 0, row 1, row 2, column 0,
 * column 1, column 2, in that order.
 */
void oracle_det_expansions(const double* z, int64_t n, int64_t ld, double* out)
{
    for (int64_t p = 0; p < n; ++p) {
        mat3 A = unpack(z, ld, p);
        for (int k = 0; k < 3; ++k) {
            cplx r = det_by_row(&A, k);
            cplx c = det_by_column(&A, k);
            out[(2 * k) * n + p] = creal(r);
            out[(2 * k + 1) * n + p] = cimag(r);
            out[(6 + 2 * k) * n + p] = creal(c);
            out[(6 + 2 * k + 1) * n + p] = cimag(c);
        }
    }
}

/*
 * Full 3x3 inverse, row-major complex: out[(2*(3*i+j)) * n + p] = Re X[i][j],
 * out[(2*(3*i+j)+1) * n + p] = Im X[i][j].  method 0: Gauss-Jordan; method 1:
 * adj/det (Eq. inv_adjoint).
 */
void oracle_inverse_full(const double* z, int64_t n, int64_t ld, int method, double* out)
{
    for (int64_t p = 0; p < n; ++p) {
        mat3 A = unpack(z, ld, p), X;
        if (method == 1) {
            adj_inverse(&A, &X);
        } else if (ge_inverse(&A, &X) != 0) {
            fill_nan(out, n, p, 18);
            continue;
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                out[(2 * (3 * i + j)) * n + p] = creal(X.m[i][j]);
                out[(2 * (3 * i + j) + 1) * n + p] = cimag(X.m[i][j]);
            }
    }
}

/* lam: [3][n] ascending eigenvalues of each pixel's Hermitian Z. */
void oracle_eigvals(const double* z, int64_t n, int64_t ld, double* lam)
{
    for (int64_t p = 0; p < n; ++p) {
        mat3 A = unpack(z, ld, p);
        double l[3];
        jacobi_eigvals(&A, l);
        lam[0 * n + p] = l[0];
        lam[1 * n + p] = l[1];
        lam[2 * n + p] = l[2];
    }
}

/* ------------------------------------------------------------------------ */
/* Multilook covariance (Eq. ZN) over a window, clamp-to-edge addressing     */
/* ------------------------------------------------------------------------ */

static int64_t clampi(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

static cplx slc(const double* s, int64_t plane_ld, int64_t W, int comp, int64_t y, int64_t x)
{
    const double* q = s + 2 * (comp * plane_ld + y * W + x);
    return q[0] + I * q[1];
}

/*
 * Z at pixel (y, x): sum over the window offsets (dy, dx) in [-r, r]^2, r =
 * (win-1)/2, of w[(dy+r)*win + (dx+r)] * S S^H with S = s(clamp(y+dy), clamp(x+dx)).
 * w == NULL means the boxcar average of Eq. ZN: the plain sum divided by N = win^2.
 */
static mat3 window_cov(const double* s, int64_t H, int64_t W, int64_t plane_ld, int win,
                       const double* w, int64_t y, int64_t x)
{
    int r = (win - 1) / 2;
    mat3 Z;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Z.m[i][j] = 0.0;
    for (int dy = -r; dy <= r; ++dy) {
        for (int dx = -r; dx <= r; ++dx) {
#if ORACLE_MUTANT == 5
            int64_t yy = clampi(y + dy, 0, H - 2); /* mutant: wrong clamp bound */
#else
            int64_t yy = clampi(y + dy, 0, H - 1);
#endif
            int64_t xx = clampi(x + dx, 0, W - 1);
            double wk = w ? w[(dy + r) * win + (dx + r)] : 1.0;
            cplx S[3];
            for (int i = 0; i < 3; ++i) S[i] = slc(s, plane_ld, W, i, yy, xx);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
#if ORACLE_MUTANT == 4
                    Z.m[i][j] += wk * S[i] * S[j]; /* mutant: conjugation dropped */
#else
                    Z.m[i][j] += wk * S[i] * conj(S[j]);
#endif
        }
    }
    if (!w) {
        double N = (double)win * (double)win;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Z.m[i][j] /= N;
    }
    return Z;
}

/* z: [9][H*W] packed multilook covariance. */
void oracle_multilook(const double* s, int64_t H, int64_t W, int64_t plane_ld, int win,
                      const double* w, double* z)
{
    int64_t n = H * W;
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            mat3 Z = window_cov(s, H, W, plane_ld, win, w, y, x);
            pack_upper(&Z, z, n, y * W + x);
        }
}

/* ------------------------------------------------------------------------ */
/* Gradient of a per-pixel loss L(W = Z^-1, det Z, log det Z) w.r.t. the     */
/* nine packed reals of Z.                                                  */
/*                                                                          */
/* Upstream packed gradients g (one real per packed plane of W) define the  */
/* Hermitian G with G_ii = g_ii and G_ij = (g_Re + i g_Im)/2 (i < j), so    */
/* that sum_k g_k dW_k = Re tr(G dW).  With dW = -W dZ W,                   */
/* d det = det tr(W dZ) and d log det = tr(W dZ):                           */
/*     dL = Re tr(M dZ),  M = -W G W + (g_det det + g_logdet) W,            */
/* and the packed gradient is [M00, 2Re M01, 2Im M01, 2Re M02, 2Im M02,     */
/* M11, 2Re M12, 2Im M12, M22].                                             */
/* ------------------------------------------------------------------------ */

static mat3 hermitian_from_packed_grad(const double* g, int64_t n, int64_t p)
{
    mat3 G;
    cplx b = 0.5 * (g[1 * n + p] + I * g[2 * n + p]);
    cplx c = 0.5 * (g[3 * n + p] + I * g[4 * n + p]);
    cplx e = 0.5 * (g[6 * n + p] + I * g[7 * n + p]);
    G.m[0][0] = g[0 * n + p];
    G.m[1][1] = g[5 * n + p];
    G.m[2][2] = g[8 * n + p];
    G.m[0][1] = b;
    G.m[1][0] = conj(b);
    G.m[0][2] = c;
    G.m[2][0] = conj(c);
    G.m[1][2] = e;
    G.m[2][1] = conj(e);
    return G;
}

static void pack_grad(const mat3* M, double* out, int64_t n, int64_t p)
{
#if ORACLE_MUTANT == 6
    double two = 1.0; /* mutant: off-diagonal factor 2 dropped */
#else
    double two = 2.0;
#endif
    out[0 * n + p] = creal(M->m[0][0]);
    out[1 * n + p] = two * creal(M->m[0][1]);
    out[2 * n + p] = two * cimag(M->m[0][1]);
    out[3 * n + p] = two * creal(M->m[0][2]);
    out[4 * n + p] = two * cimag(M->m[0][2]);
    out[5 * n + p] = creal(M->m[1][1]);
    out[6 * n + p] = two * creal(M->m[1][2]);
    out[7 * n + p] = two * cimag(M->m[1][2]);
    out[8 * n + p] = creal(M->m[2][2]);
}

/*
 * z: [9][ld] packed input; g_zinv: [9][n] or NULL; g_det, g_logdet: [n] or NULL;
 * g_z: [9][n] output.
 */
void oracle_zinv_det_bwd(const double* z, int64_t n, int64_t ld, const double* g_zinv,
                         const double* g_det, const double* g_logdet, double* g_z)
{
    for (int64_t p = 0; p < n; ++p) {
        mat3 A = unpack(z, ld, p), W;
        if (ge_inverse(&A, &W) != 0) {
            fill_nan(g_z, n, p, 9);
            continue;
        }
        double det = creal(det_ge(&A));
        double s = 0.0;
        if (g_det) s += g_det[p] * det;
        if (g_logdet) s += g_logdet[p];
        mat3 M;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M.m[i][j] = s * W.m[i][j];
        if (g_zinv) {
            mat3 G = hermitian_from_packed_grad(g_zinv, n, p), WG, WGW;
            matmul3(&W, &G, &WG);
            matmul3(&WG, &W, &WGW);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
#if ORACLE_MUTANT == 10
                    M.m[i][j] += WGW.m[i][j]; /* mutant: sign of the inverse term */
#else
                    M.m[i][j] -= WGW.m[i][j];
#endif
        }
        pack_grad(&M, g_z, n, p);
    }
}

/* ------------------------------------------------------------------------ */
/* Wishart change statistic between two dates (the likelihood-ratio test    */
/* of §1).  Per pixel, with Z_t the weighted window covariance of date t:    */
/*     q = ln det Z1 + ln det Z2 - 2 ln det((Z1 + Z2) / 2)                   */
/* and the loss L = sum_p q(p).  q <= 0 with equality iff Z1 = Z2.           */
/* ------------------------------------------------------------------------ */

static double logdet(const mat3* A)
{
    return log(creal(det_ge(A)));
}

static double wishart_q(const mat3* Z1, const mat3* Z2)
{
    mat3 Zm;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
#if ORACLE_MUTANT == 7
            Zm.m[i][j] = Z1->m[i][j] + Z2->m[i][j]; /* mutant: the 1/2 dropped */
#else
            Zm.m[i][j] = 0.5 * (Z1->m[i][j] + Z2->m[i][j]);
#endif
    return logdet(Z1) + logdet(Z2) - 2.0 * logdet(&Zm);
}

/* q_map: [H*W] or NULL; loss: scalar sum of q over all pixels. */
void oracle_wishart_fwd(const double* s1, const double* s2, int64_t H, int64_t W,
                        int64_t plane_ld, int win, const double* w, double* q_map,
                        double* loss)
{
    double L = 0.0;
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            mat3 Z1 = window_cov(s1, H, W, plane_ld, win, w, y, x);
            mat3 Z2 = window_cov(s2, H, W, plane_ld, win, w, y, x);
            double q = wishart_q(&Z1, &Z2);
            if (q_map) q_map[y * W + x] = q;
            L += q;
        }
    *loss = L;
}

/*
 * grad_w[k] = g * dL/dw_k.  With W_t = Z_t^-1 and W_12 = (Z1 + Z2)^-1,
 * dq = tr(M1 dZ1) + tr(M2 dZ2), M_t = W_t - 2 W_12, and dZ_t(p)/dw_k =
 * S S^H with S = s_t(clamp(p + offset_k)), so dL/dw_k = sum_p sum_t S^H M_t(p) S.
 */
void oracle_wishart_bwd_rows(const double* s1, const double* s2, int64_t H, int64_t W,
                             int64_t plane_ld, int win, const double* w, double g, int64_t y_lo,
                             int64_t y_hi, double* grad_w)
{
    int r = (win - 1) / 2;
    int K = win * win;
    for (int k = 0; k < K; ++k) grad_w[k] = 0.0;
    const double* s_t[2] = {s1, s2};
    for (int64_t y = y_lo; y < y_hi; ++y)
        for (int64_t x = 0; x < W; ++x) {
            mat3 Z[2], Wt[2], Z12, W12;
            Z[0] = window_cov(s1, H, W, plane_ld, win, w, y, x);
            Z[1] = window_cov(s2, H, W, plane_ld, win, w, y, x);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Z12.m[i][j] = Z[0].m[i][j] + Z[1].m[i][j];
            if (ge_inverse(&Z[0], &Wt[0]) || ge_inverse(&Z[1], &Wt[1]) ||
                ge_inverse(&Z12, &W12)) {
                for (int k = 0; k < K; ++k) grad_w[k] = NAN;
                return;
            }
            for (int t = 0; t < 2; ++t) {
                mat3 M;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
#if ORACLE_MUTANT == 8
                        M.m[i][j] = Wt[t].m[i][j] - W12.m[i][j]; /* mutant: factor 2 dropped */
#else
                        M.m[i][j] = Wt[t].m[i][j] - 2.0 * W12.m[i][j];
#endif
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx) {
                        int64_t yy = clampi(y + dy, 0, H - 1);
                        int64_t xx = clampi(x + dx, 0, W - 1);
                        cplx S[3];
                        for (int i = 0; i < 3; ++i)
                            S[i] = slc(s_t[t], plane_ld, W, i, yy, xx);
                        cplx quad = 0;
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) quad += conj(S[i]) * M.m[i][j] * S[j];
                        grad_w[(dy + r) * win + (dx + r)] += g * creal(quad);
                    }
            }
        }
}

void oracle_wishart_bwd(const double* s1, const double* s2, int64_t H, int64_t W,
                        int64_t plane_ld, int win, const double* w, double g, double* grad_w)
{
    oracle_wishart_bwd_rows(s1, s2, H, W, plane_ld, win, w, g, 0, H, grad_w);
}

/* ------------------------------------------------------------------------ */
/* Nonlocal-means filter with a stochastic distance (§1: the paper's         */
/* motivating workload, 23 x 23 search windows).  For pixels i, j with       */
/* covariances Z_i, Z_j of the same number of looks L:                       */
/*     d(i, j) = ln det((Z_i + Z_j)/2) - (ln det Z_i + ln det Z_j)/2  (>= 0), */
/* the Wishart equal-looks statistic (half the negative log-likelihood ratio */
/* q of the change test, per look); weights w_ij = exp(-L d(i, j) / h) over  */
/* the neighbours j inside the image within the search radius, and           */
/*     Z'_i = sum_j w_ij Z_j / sum_j w_ij.                                   */
/* ------------------------------------------------------------------------ */

double oracle_pair_distance(const double* zi, const double* zj)
{
    mat3 A = unpack(zi, 1, 0), B = unpack(zj, 1, 0), M;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M.m[r][c] = 0.5 * (A.m[r][c] + B.m[r][c]);
    return logdet(&M) - 0.5 * (logdet(&A) + logdet(&B));
}

void oracle_nlm_wishart(const double* z, int64_t H, int64_t W, int radius, double looks,
                        double h, double* out)
{
    int64_t n = H * W;
    double* ld = (double*)malloc((size_t)n * sizeof(double));
    for (int64_t p = 0; p < n; ++p) {
        mat3 A = unpack(z, n, p);
        ld[p] = logdet(&A);
    }
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            int64_t i = y * W + x;
            mat3 Zi = unpack(z, n, i);
            double acc[9] = {0}, wsum = 0.0;
            for (int dy = -radius; dy <= radius; ++dy)
                for (int dx = -radius; dx <= radius; ++dx) {
                    int64_t yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    int64_t j = yy * W + xx;
                    mat3 Zj = unpack(z, n, j), M;
#if ORACLE_MUTANT == 12
                    double half = 1.0; /* mutant: pair mean without the 1/2 */
#else
                    double half = 0.5;
#endif
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c) M.m[r][c] = half * (Zi.m[r][c] + Zj.m[r][c]);
                    double d = logdet(&M) - 0.5 * (ld[i] + ld[j]);
                    double w = exp(-looks * d / h);
                    for (int k = 0; k < 9; ++k) acc[k] += w * z[k * n + j];
                    wsum += w;
                }
            for (int k = 0; k < 9; ++k) out[k * n + i] = acc[k] / wsum;
        }
    free(ld);
}

/* ------------------------------------------------------------------------ */
/* Stochastic distances between the complex Wishart laws W(S_i, L) and      */
/* W(S_j, L) of two pixels with the same number of looks L and m = 3 (§1     */
/* lists Kullback-Leibler, Hellinger, Renyi, Bhattacharyya, triangular and   */
/* harmonic divergences among the uses of det Z and Z^-1).  From the density */
/*     f(Z) = c(L) |Z|^(L-m) |S|^-L exp(-L tr(S^-1 Z)),  E[Z] = S:           */
/*   Bhattacharyya  d_B = -ln of the integral of sqrt(f_i f_j)               */
/*                      = L [ln det((S_i^-1 + S_j^-1)/2)                     */
/*                           + (ln det S_i + ln det S_j)/2],                 */
/*   Hellinger      d_H = 1 - that integral = 1 - exp(-d_B),                 */
/*   Kullback-Leibler (the mean of the two directed divergences)             */
/*                  d_KL = L [(tr(S_i^-1 S_j) + tr(S_j^-1 S_i))/2 - m],      */
/*   Renyi of order b in (0, 1) (the mean of the two directed divergences    */
/*   D_b(i||j) = ln(integral of f_i^b f_j^(1-b)) / (b - 1))                  */
/*                  D_b(i||j) = L/(1-b) [ln det(b S_i^-1 + (1-b) S_j^-1)     */
/*                                       + b ln det S_i + (1-b) ln det S_j]. */
/* All four are >= 0, symmetric, and 0 iff S_i = S_j.  The oracle takes      */
/* them as written, with Gauss-Jordan inverses and elimination dets.         */
/* ------------------------------------------------------------------------ */

#define ORACLE_DIST_BHATTACHARYYA 0
#define ORACLE_DIST_HELLINGER 1
#define ORACLE_DIST_KULLBACK_LEIBLER 2
#define ORACLE_DIST_RENYI 3

/* tr(X Y) = sum_r sum_c X[r][c] Y[c][r] (real for Hermitian X, Y). */
static double trace_of_product(const mat3* X, const mat3* Y)
{
    cplx t = 0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
#if ORACLE_MUTANT == 13
            t += X->m[r][c] * Y->m[r][c]; /* mutant: Y's element not transposed */
#else
            t += X->m[r][c] * Y->m[c][r];
#endif
    return creal(t);
}

/* Directed Renyi divergence of order b of W(S_x, L) from W(S_y, L), from the
 * inverses Ix, Iy and log-dets of S_x, S_y. */
static double renyi_directed(const mat3* Ix, const mat3* Iy, double ldx, double ldy,
                             double looks, double b)
{
    mat3 A;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
#if ORACLE_MUTANT == 15
            A.m[r][c] = b * (Ix->m[r][c] + Iy->m[r][c]); /* mutant: b on both terms */
#else
            A.m[r][c] = b * Ix->m[r][c] + (1.0 - b) * Iy->m[r][c];
#endif
    return looks / (1.0 - b) * (logdet(&A) + b * ldx + (1.0 - b) * ldy);
}

/* One pixel pair, given both covariances, their inverses and log-dets. */
static double stochastic_distance(const mat3* Si, const mat3* Sj, const mat3* Ii,
                                  const mat3* Ij, double ldi, double ldj, double looks,
                                  int dist, double order)
{
    if (dist == ORACLE_DIST_KULLBACK_LEIBLER)
        return looks * (0.5 * (trace_of_product(Ii, Sj) + trace_of_product(Ij, Si)) - 3.0);
    if (dist == ORACLE_DIST_RENYI)
        return 0.5 * (renyi_directed(Ii, Ij, ldi, ldj, looks, order) +
                      renyi_directed(Ij, Ii, ldj, ldi, looks, order));
    mat3 M;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M.m[r][c] = 0.5 * (Ii->m[r][c] + Ij->m[r][c]);
    double dB = looks * (logdet(&M) + 0.5 * (ldi + ldj));
    if (dist == ORACLE_DIST_HELLINGER)
#if ORACLE_MUTANT == 14
        return 1.0 - exp(-0.5 * dB); /* mutant: square root of the coefficient */
#else
        return 1.0 - exp(-dB);
#endif
    return dB;
}

/* d(S_i, S_j) for packed zi, zj (nine doubles each); `order` is the Renyi
 * order b in (0, 1), unused by the other distances.  NaN for an unknown dist,
 * an order outside (0, 1) for Renyi, or a singular matrix. */
double oracle_stochastic_distance(const double* zi, const double* zj, double looks, int dist,
                                  double order)
{
    if (dist < 0 || dist > 3) return NAN;
    if (dist == ORACLE_DIST_RENYI && !(order > 0.0 && order < 1.0)) return NAN;
    mat3 Si = unpack(zi, 1, 0), Sj = unpack(zj, 1, 0), Ii, Ij;
    if (ge_inverse(&Si, &Ii) || ge_inverse(&Sj, &Ij)) return NAN;
    return stochastic_distance(&Si, &Sj, &Ii, &Ij, logdet(&Si), logdet(&Sj), looks, dist,
                               order);
}

/* Nonlocal means with weights w_ij = exp(-d(i, j) / h) over the in-image
 * neighbours within the search radius (d including the factor L); the
 * Bhattacharyya case equals oracle_nlm_wishart. */
void oracle_nlm_stochastic(const double* z, int64_t H, int64_t W, int radius, double looks,
                           double h, int dist, double order, double* out)
{
    int64_t n = H * W;
    mat3* inv = (mat3*)malloc((size_t)n * sizeof(mat3));
    double* ld = (double*)malloc((size_t)n * sizeof(double));
    for (int64_t p = 0; p < n; ++p) {
        mat3 A = unpack(z, n, p);
        ld[p] = logdet(&A);
        if (ge_inverse(&A, &inv[p])) ld[p] = NAN;
    }
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            int64_t i = y * W + x;
            mat3 Si = unpack(z, n, i);
            double acc[9] = {0}, wsum = 0.0;
            for (int dy = -radius; dy <= radius; ++dy)
                for (int dx = -radius; dx <= radius; ++dx) {
                    int64_t yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    int64_t j = yy * W + xx;
                    mat3 Sj = unpack(z, n, j);
                    double d = stochastic_distance(&Si, &Sj, &inv[i], &inv[j], ld[i], ld[j],
                                                   looks, dist, order);
                    double w = exp(-d / h);
                    for (int k = 0; k < 9; ++k) acc[k] += w * z[k * n + j];
                    wsum += w;
                }
            for (int k = 0; k < 9; ++k) out[k * n + i] = acc[k] / wsum;
        }
    free(ld);
    free(inv);
}

/* ------------------------------------------------------------------------ */
/* Multifrequency data (§5): per pixel a block-diagonal Hermitian matrix of  */
/* nb 3x3 Hermitian blocks.  The oracle inverts the full 3nb x 3nb matrix by */
/* Gauss-Jordan elimination with partial pivoting and takes its det from     */
/* the pivots -- the plain definition, which does not use the block         */
/* structure -- and returns the diagonal blocks of the inverse (packed) and  */
/* the largest modulus found off the diagonal blocks (zero in exact          */
/* arithmetic).                                                             */
/* ------------------------------------------------------------------------ */

#define ORACLE_MAX_BLOCKS 8

static int ge_inverse_n(int m, const cplx* A, cplx* X, cplx* det)
{
    cplx M[3 * ORACLE_MAX_BLOCKS][6 * ORACLE_MAX_BLOCKS];
    cplx prod = 1.0;
    int swaps = 0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            M[i][j] = A[i * m + j];
            M[i][m + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (cabs(M[r][col]) > cabs(M[piv][col])) piv = r;
        if (cabs(M[piv][col]) == 0.0) {
            *det = 0.0;
            return -1;
        }
        if (piv != col) {
            ++swaps;
            for (int k = 0; k < 2 * m; ++k) {
                cplx t = M[col][k];
                M[col][k] = M[piv][k];
                M[piv][k] = t;
            }
        }
        prod *= M[col][col];
        cplx inv_p = 1.0 / M[col][col];
        for (int k = 0; k < 2 * m; ++k) M[col][k] *= inv_p;
        for (int r = 0; r < m; ++r) {
            if (r == col) continue;
            cplx factor = M[r][col];
            for (int k = 0; k < 2 * m; ++k) M[r][k] -= factor * M[col][k];
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) X[i * m + j] = M[i][m + j];
    *det = (swaps % 2) ? -prod : prod;
    return 0;
}

/*
 * z: [nb][9][ld] packed blocks; zinv: [nb][9][n] packed diagonal blocks of the
 * full inverse; det: [n] det of the full matrix; off: [n] max |entry| of the
 * full inverse outside the diagonal blocks.
 */
void oracle_zinv_det_blockdiag(const double* z, int nb, int64_t n, int64_t ld, double* zinv,
                               double* det, double* off)
{
    int m = 3 * nb;
    cplx A[9 * ORACLE_MAX_BLOCKS * ORACLE_MAX_BLOCKS], X[9 * ORACLE_MAX_BLOCKS * ORACLE_MAX_BLOCKS];
    for (int64_t p = 0; p < n; ++p) {
        for (int i = 0; i < m * m; ++i) A[i] = 0.0;
        for (int b = 0; b < nb; ++b) {
            mat3 B = unpack(z + (int64_t)b * 9 * ld, ld, p);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) A[(3 * b + i) * m + 3 * b + j] = B.m[i][j];
        }
        cplx dt;
        if (ge_inverse_n(m, A, X, &dt) != 0) {
            for (int b = 0; b < nb; ++b) fill_nan(zinv + (int64_t)b * 9 * n, n, p, 9);
            det[p] = 0.0;
            off[p] = NAN;
            continue;
        }
        det[p] = creal(dt);
        double mx = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j)
                if (i / 3 != j / 3 && cabs(X[i * m + j]) > mx) mx = cabs(X[i * m + j]);
        off[p] = mx;
        for (int b = 0; b < nb; ++b) {
            mat3 Y;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Y.m[i][j] = X[(3 * b + i) * m + 3 * b + j];
            pack_upper(&Y, zinv + (int64_t)b * 9 * n, n, p);
        }
    }
}
