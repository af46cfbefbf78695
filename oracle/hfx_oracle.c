/*
 * hfx_oracle.c -- plain, slow, FP64 CPU oracle for the nonlocal
 * Hartree-Fock exchange matrix of Betzinger, Friedrich and Bluegel,
 * "Hybrid functionals within the all-electron FLAPW method" (Sec. III).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check and the CPU-baseline leg of
 * bench.py do.  It shares no code, header, table or constant with the CUDA
 * library: every formula below is written out from the paper's definitions.
 *
 * Every function states the passage it follows.  Loops are direct sums over
 * the indices of the definition; OpenMP only distributes independent (k,q)
 * pairs of the Brillouin-zone sum over host threads.
 *
 * Parity pins (tests/test_oracle_*.py) tie each function to something other
 * than itself: 3-j closed forms and numerical quadrature of spherical
 * harmonics (Gaunt), radial quadrature of the sphere Fourier transform and a
 * real-space brute force of the interstitial integral (step function and
 * Z^IPW), a 3-D quadrature of the muffin-tin triple product (Z^MT),
 * orthogonality and invariance (multipole transform), Hermiticity,
 * negative semi-definiteness and a literal four-index sum (V^x), the
 * analytic integral behind Eq. (div final), and the exchange-energy identity.
 *
 * Conventions: complex numbers are interleaved double pairs; see the python
 * binding oracle/oracle.py for array shapes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) { cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static inline cplx cconjmul(cplx a, cplx b) { /* conj(a) * b */ cplx r = {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re}; return r; }
static inline cplx cconj(cplx a) { cplx r = {a.re, -a.im}; return r; }
static inline cplx cadd(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cplx cscale(cplx a, double s) { cplx r = {a.re * s, a.im * s}; return r; }

/* All inputs of one build.  Pointers are borrowed (owned by the caller). */
typedef struct {
    double lattice[9];          /* rows a_i, bohr */
    int n_atoms;
    const double *pos_frac;     /* [n_atoms][3] */
    const double *rmt;          /* [n_atoms] */
    int lmax, Lmax, P;
    int mesh[3];
    const int *n_bands;         /* [N_k] */
    const int *n_occ;           /* [N_k] */
    const int *npw;             /* [N_k] */
    const long long *pw_off;    /* [N_k] row offset into Gk */
    const int *Gk;              /* [sum npw][3] */
    const long long *c_off;     /* [N_k] complex offset into c */
    const double *c;            /* per k: [n_bands][npw] complex */
    const long long *A_off;     /* [N_k] complex offset into A */
    const double *A;            /* per k: [n_bands][n_atoms][N_lmp] complex */
    const double *R;            /* [n_atoms][(Lmax+1)P][2(lmax+1)][2(lmax+1)] */
    const double *mu;           /* [n_atoms][(Lmax+1)P] */
    const int *n_ipw;           /* [N_k] per q */
    const long long *gaux_off;  /* [N_k] row offset into Gaux */
    const int *Gaux;            /* [sum n_ipw][3] */
    const long long *v_off;     /* [N_k] complex offset into v */
    const double *v;            /* per q: [N_aux][N_aux] complex, row-major */
    double beta;
} OraSys;

/* ---------------------------------------------------------------- geometry */

static double det3(const double *m) {
    return m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
           m[2] * (m[3] * m[7] - m[4] * m[6]);
}

/* Unit-cell volume Omega (Eq. FLAPW-basis normalisation). */
double ora_omega(const OraSys *s) { return fabs(det3(s->lattice)); }

/* Reciprocal rows b_i with a_i . b_j = 2 pi delta_ij. */
static void recip(const OraSys *s, double *B) {
    const double *a = s->lattice;
    double det = det3(a);
    /* B = 2 pi (A^{-1})^T ; (A^{-1})^T = cofactor(A) / det */
    double cof[9];
    cof[0] = a[4] * a[8] - a[5] * a[7];
    cof[1] = -(a[3] * a[8] - a[5] * a[6]);
    cof[2] = a[3] * a[7] - a[4] * a[6];
    cof[3] = -(a[1] * a[8] - a[2] * a[7]);
    cof[4] = a[0] * a[8] - a[2] * a[6];
    cof[5] = -(a[0] * a[7] - a[1] * a[6]);
    cof[6] = a[1] * a[5] - a[2] * a[4];
    cof[7] = -(a[0] * a[5] - a[2] * a[3]);
    cof[8] = a[0] * a[4] - a[1] * a[3];
    for (int i = 0; i < 9; ++i) B[i] = 2.0 * M_PI * cof[i] / det;
}

static int n_k(const OraSys *s) { return s->mesh[0] * s->mesh[1] * s->mesh[2]; }

static void mesh_j(const OraSys *s, int ik, int *j) {
    j[2] = ik % s->mesh[2];
    j[1] = (ik / s->mesh[2]) % s->mesh[1];
    j[0] = ik / (s->mesh[1] * s->mesh[2]);
}

/* Sec. III.C: the mesh contains k - q.  For a pair (k, q) return k' = k - q
 * folded into the mesh and the reciprocal vector G0 = k - q - k' (integer
 * coordinates in units of b_i). */
void ora_fold(const OraSys *s, int ik, int iq, int *ikp, int *G0) {
    int jk[3], jq[3], jp[3];
    mesh_j(s, ik, jk);
    mesh_j(s, iq, jq);
    for (int i = 0; i < 3; ++i) {
        int d = jk[i] - jq[i];
        int f = ((d % s->mesh[i]) + s->mesh[i]) % s->mesh[i];
        jp[i] = f;
        G0[i] = (d - f) / s->mesh[i];
    }
    *ikp = (jp[0] * s->mesh[1] + jp[1]) * s->mesh[2] + jp[2];
}

static void cart_of(const double *B, const double *frac, double *out) {
    for (int x = 0; x < 3; ++x) out[x] = frac[0] * B[0 * 3 + x] + frac[1] * B[1 * 3 + x] + frac[2] * B[2 * 3 + x];
}

/* ---------------------------------------------------------------- Gaunt */

static double fact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* Wigner 3-j symbol from Racah's closed formula. */
double ora_threej(int j1, int j2, int j3, int m1, int m2, int m3) {
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
    /* (j1 j2 j3; 0 0 0) vanishes for odd j1 + j2 + j3 (reflection symmetry) */
    if (m1 == 0 && m2 == 0 && ((j1 + j2 + j3) & 1)) return 0.0;
    double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
    double pre = sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                      fact(j3 + m3) * fact(j3 - m3));
    double sum = 0.0;
    for (int t = 0; t <= j1 + j2 + j3; ++t) {
        int a1 = j3 - j2 + t + m1, a2 = j3 - j1 + t - m2, a3 = j1 + j2 - j3 - t;
        int a4 = j1 - t - m1, a5 = j2 - t + m2;
        if (a1 < 0 || a2 < 0 || a3 < 0 || a4 < 0 || a5 < 0) continue;
        double den = fact(t) * fact(a1) * fact(a2) * fact(a3) * fact(a4) * fact(a5);
        sum += ((t & 1) ? -1.0 : 1.0) / den;
    }
    int ph = j1 - j2 - m3;
    double sign = ((ph % 2) + 2) % 2 ? -1.0 : 1.0;
    return sign * pre * sum;
}

/* Integral of Y_{l1 m1} Y_{l2 m2} Y_{l3 m3} over the unit sphere (complex
 * Condon-Shortley harmonics; textbook 3-j form). */
static double int_yyy(int l1, int m1, int l2, int m2, int l3, int m3) {
    double w = ora_threej(l1, l2, l3, 0, 0, 0);
    if (w == 0.0) return 0.0;
    return sqrt((2.0 * l1 + 1.0) * (2.0 * l2 + 1.0) * (2.0 * l3 + 1.0) / (4.0 * M_PI)) * w *
           ora_threej(l1, l2, l3, m1, m2, m3);
}

/* G(LM; l m; l' m') = int Y*_LM Y*_lm Y_l'm' dOmega: the angular factor of
 * the MT product functions u_lp u_l'p' Y_LM (Sec. III.B).  Uses
 * Y*_lm = (-1)^m Y_{l,-m}. */
double ora_gaunt(int L, int M, int l1, int m1, int l2, int m2) {
    if (abs(M) > L || abs(m1) > l1 || abs(m2) > l2) return 0.0;
    double s = ((M + m1) & 1) ? -1.0 : 1.0;
    return s * int_yyy(L, -M, l1, -m1, l2, m2);
}

/* ---------------------------------------------------------- step function */

/* Theta_K = (1/Omega) int_cell Theta(r) e^{-i K.r} d^3r for the step function
 * of Eq. (step function): 1 in the interstitial, 0 inside every MT sphere.
 * The Fourier transform of a sphere of radius S at R_a is
 * e^{-i K.R_a} 4 pi S^3 j1(|K| S) / (|K| S). */
void ora_theta(const OraSys *s, int n, const int *K, double *out) {
    double B[9];
    recip(s, B);
    double om = ora_omega(s);
    for (int i = 0; i < n; ++i) {
        double kf[3] = {(double)K[3 * i], (double)K[3 * i + 1], (double)K[3 * i + 2]};
        double kc[3];
        cart_of(B, kf, kc);
        double kn = sqrt(kc[0] * kc[0] + kc[1] * kc[1] + kc[2] * kc[2]);
        int zero = (K[3 * i] == 0 && K[3 * i + 1] == 0 && K[3 * i + 2] == 0);
        cplx t = {zero ? 1.0 : 0.0, 0.0};
        for (int a = 0; a < s->n_atoms; ++a) {
            double S = s->rmt[a];
            double f;
            double x = kn * S;
            if (zero) {
                f = 4.0 * M_PI * S * S * S / 3.0;
            } else if (x < 1e-3) {
                /* j1(x)/x = 1/3 - x^2/30 + O(x^4) */
                f = 4.0 * M_PI * S * S * S * (1.0 / 3.0 - x * x / 30.0);
            } else {
                double j1 = sin(x) / (x * x) - cos(x) / x;
                f = 4.0 * M_PI * S * S * S * j1 / x;
            }
            /* phase e^{-i K.R_a}, K.R_a = 2 pi sum_i K_i f_i */
            double ph = 2.0 * M_PI * (K[3 * i] * s->pos_frac[3 * a] + K[3 * i + 1] * s->pos_frac[3 * a + 1] +
                                      K[3 * i + 2] * s->pos_frac[3 * a + 2]);
            t.re -= f * cos(ph) / om;
            t.im -= -f * sin(ph) / om;
        }
        out[2 * i] = t.re;
        out[2 * i + 1] = t.im;
    }
}

/* ------------------------------------------------------- index helpers */

static int n_lmp(const OraSys *s) { return 2 * (s->lmax + 1) * (s->lmax + 1); }
static int n_lp(const OraSys *s) { return 2 * (s->lmax + 1); }
static int n_mt(const OraSys *s) { return s->n_atoms * (s->Lmax + 1) * (s->Lmax + 1) * s->P; }
static int lm_idx(int l, int m) { return l * l + l + m; }

static const cplx *cptr(const double *base, long long off) { return (const cplx *)(base + 2 * off); }

/* ------------------------------------------------------------ Z^MT */

/* Muffin-tin part of the projection vectors (Sec. III.B and Eq. vec-mat-vec):
 *   Z[(a,L,M,P), m, n] = < M^q_{aLMP} phi_{m,k-q} | phi_{n,k} >
 *     = e^{-i q.R_a} sum_{l m1 p l' p'} G(LM; l m1; l', m1+M)
 *         R^a_{LP; lp; l'p'} conj(A^a_{l m1 p}(m, k')) A^a_{l', m1+M, p'}(n, k).
 * The phase comes from the Bloch sum Eq. (MT functions) evaluated in the home
 * cell; the MT coefficients of phi_{m,k-q} are those of phi_{m,k'}.
 * Output Z[I][m][n], I over the MT product basis, m < n_occ(k'), n < n_bands(k). */
/* Bands n of the projection: sel[j] for j < nsel (all bands 0..nb-1 when sel
 * is NULL).  inner != 0 spreads the rows over the OpenMP threads. */
static void zmt_core(const OraSys *s, int ik, int iq, const int *sel, int nsel, int inner, double *Zout) {
    int ikp, G0[3];
    ora_fold(s, ik, iq, &ikp, G0);
    int nb = nsel, no = s->n_occ[ikp];
    int nlmp = n_lmp(s), nlp = n_lp(s), P = s->P;
    int nLP = (s->Lmax + 1) * P;
    int nlm = (s->lmax + 1) * (s->lmax + 1), nLM = (s->Lmax + 1) * (s->Lmax + 1);
    /* Gaunt values G(LM; l m1; l2, m1+M), tabulated once per call */
    double *gt = (double *)malloc(sizeof(double) * nLM * nlm * (s->lmax + 1));
    for (int L = 0; L <= s->Lmax; ++L)
        for (int M = -L; M <= L; ++M)
            for (int l = 0; l <= s->lmax; ++l)
                for (int m1 = -l; m1 <= l; ++m1)
                    for (int l2 = 0; l2 <= s->lmax; ++l2)
                        gt[((size_t)lm_idx(L, M) * nlm + lm_idx(l, m1)) * (s->lmax + 1) + l2] =
                            ora_gaunt(L, M, l, m1, l2, m1 + M);
    int jq[3];
    mesh_j(s, iq, jq);
    double qf[3] = {(double)jq[0] / s->mesh[0], (double)jq[1] / s->mesh[1], (double)jq[2] / s->mesh[2]};
    const cplx *Ak = cptr(s->A, s->A_off[ik]);
    const cplx *Akp = cptr(s->A, s->A_off[ikp]);
    cplx *Z = (cplx *)Zout;
    const int nI = s->n_atoms * nLM * P;
#pragma omp parallel for schedule(dynamic) if (inner)
    for (int I = 0; I < nI; ++I) {
        const int a = I / (nLM * P), LM = (I / P) % nLM, Pi = I % P;
        const int L = (int)floor(sqrt((double)LM) + 1e-9), M = LM - L * L - L;
        /* e^{-i q.R_a}, q.R_a = 2 pi sum_i qf_i f_i */
        double ph = 2.0 * M_PI * (qf[0] * s->pos_frac[3 * a] + qf[1] * s->pos_frac[3 * a + 1] + qf[2] * s->pos_frac[3 * a + 2]);
        cplx phase = {cos(ph), -sin(ph)};
        const double *Rap = s->R + ((size_t)a * nLP + (size_t)L * P + Pi) * nlp * nlp;
        for (int m = 0; m < no; ++m)
            for (int n = 0; n < nb; ++n) {
                cplx acc = {0.0, 0.0};
                for (int l = 0; l <= s->lmax; ++l)
                    for (int m1 = -l; m1 <= l; ++m1)
                        for (int p = 0; p < 2; ++p)
                            for (int l2 = 0; l2 <= s->lmax; ++l2) {
                                int m2 = m1 + M;
                                if (m2 < -l2 || m2 > l2) continue;
                                double g = gt[((size_t)lm_idx(L, M) * nlm + lm_idx(l, m1)) * (s->lmax + 1) + l2];
                                if (g == 0.0) continue;
                                for (int p2 = 0; p2 < 2; ++p2) {
                                    double r = Rap[(2 * l + p) * nlp + 2 * l2 + p2];
                                    cplx am = Akp[((size_t)m * s->n_atoms + a) * nlmp + 2 * lm_idx(l, m1) + p];
                                    const int nn = sel ? sel[n] : n;
                                    cplx an = Ak[((size_t)nn * s->n_atoms + a) * nlmp + 2 * lm_idx(l2, m2) + p2];
                                    acc = cadd(acc, cscale(cconjmul(am, an), g * r));
                                }
                            }
                Z[((size_t)I * no + m) * nb + n] = cmul(phase, acc);
            }
    }
    free(gt);
}

int ora_zmt(const OraSys *s, int ik, int iq, double *Zout) {
    zmt_core(s, ik, iq, NULL, s->n_bands[ik], 0, Zout);
    return 0;
}

/* ------------------------------------------------------------ Z^IPW */

/* Interstitial part, definition (Sec. III.B, IPW functions and Eq. step
 * function, with the wave functions of Eq. FLAPW-basis):
 *   Z[G, m, n] = < M^q_G phi_{m,k-q} | phi_{n,k} >
 *     = Omega^{-1/2} sum_{G1 in k'} sum_{G2 in k} conj(c_{G1}(m,k')) c_{G2}(n,k)
 *         Theta_{G + G1 - G2 - G0},   G0 = k - q - k'.
 * Direct triple sum; used on small inputs. */
int ora_zipw_direct(const OraSys *s, int ik, int iq, double *Zout) {
    int ikp, G0[3];
    ora_fold(s, ik, iq, &ikp, G0);
    int nb = s->n_bands[ik], no = s->n_occ[ikp];
    int npk = s->npw[ik], npp = s->npw[ikp], ng = s->n_ipw[iq];
    const int *Gk = s->Gk + 3 * s->pw_off[ik];
    const int *Gp = s->Gk + 3 * s->pw_off[ikp];
    const int *Ga = s->Gaux + 3 * s->gaux_off[iq];
    const cplx *ck = cptr(s->c, s->c_off[ik]);
    const cplx *cp = cptr(s->c, s->c_off[ikp]);
    double rs = 1.0 / sqrt(ora_omega(s));
    cplx *Z = (cplx *)Zout;
    for (int g = 0; g < ng; ++g) {
        for (int m = 0; m < no; ++m)
            for (int n = 0; n < nb; ++n) {
                cplx acc = {0.0, 0.0};
                for (int i1 = 0; i1 < npp; ++i1)
                    for (int i2 = 0; i2 < npk; ++i2) {
                        int K[3];
                        for (int x = 0; x < 3; ++x) K[x] = Ga[3 * g + x] + Gp[3 * i1 + x] - Gk[3 * i2 + x] - G0[x];
                        double th[2];
                        ora_theta(s, 1, K, th);
                        cplx t = {th[0], th[1]};
                        cplx prod = cconjmul(cp[(size_t)m * npp + i1], ck[(size_t)n * npk + i2]);
                        acc = cadd(acc, cmul(prod, t));
                    }
                Z[((size_t)g * no + m) * nb + n] = cscale(acc, rs);
            }
    }
    return 0;
}

/* The same quantity organised in the two steps of the survey's hot path:
 * first the step-function-weighted wave function in reciprocal space,
 *   T_n(K) = sum_{G2 in k} Theta_{K - G2} c_{G2}(n,k),
 * then Z[G, m, n] = Omega^{-1/2} sum_{G1 in k'} conj(c_{G1}(m,k')) T_n(G + G1 - G0).
 * T_n is evaluated on demand for each needed K (no tables), so this function
 * differs from the direct sum only in the order of the two finite sums. */
typedef struct { int lo[3], dim[3]; cplx *T; } ThetaPsi;

static void thetapsi_build(const OraSys *s, int ik, const int *lo, const int *hi, const int *sel, int nsel, ThetaPsi *tp) {
    int nb = nsel, npk = s->npw[ik];
    const int *Gk = s->Gk + 3 * s->pw_off[ik];
    const cplx *ck = cptr(s->c, s->c_off[ik]);
    for (int x = 0; x < 3; ++x) { tp->lo[x] = lo[x]; tp->dim[x] = hi[x] - lo[x] + 1; }
    size_t nbox = (size_t)tp->dim[0] * tp->dim[1] * tp->dim[2];
    tp->T = (cplx *)calloc(nbox * nb, sizeof(cplx));
    /* step function on the difference box K - G2 */
    int dlo[3], dhi[3];
    for (int x = 0; x < 3; ++x) {
        int gmin = 1 << 30, gmax = -(1 << 30);
        for (int i = 0; i < npk; ++i) { if (Gk[3 * i + x] < gmin) gmin = Gk[3 * i + x]; if (Gk[3 * i + x] > gmax) gmax = Gk[3 * i + x]; }
        dlo[x] = lo[x] - gmax;
        dhi[x] = hi[x] - gmin;
    }
    int dd[3] = {dhi[0] - dlo[0] + 1, dhi[1] - dlo[1] + 1, dhi[2] - dlo[2] + 1};
    size_t nd = (size_t)dd[0] * dd[1] * dd[2];
    int *Kd = (int *)malloc(nd * 3 * sizeof(int));
    double *th = (double *)malloc(nd * 2 * sizeof(double));
    for (size_t i = 0; i < nd; ++i) {
        int z = (int)(i % dd[2]), y = (int)((i / dd[2]) % dd[1]), xx = (int)(i / ((size_t)dd[1] * dd[2]));
        Kd[3 * i] = dlo[0] + xx; Kd[3 * i + 1] = dlo[1] + y; Kd[3 * i + 2] = dlo[2] + z;
    }
    ora_theta(s, (int)nd, Kd, th);
#pragma omp parallel for schedule(dynamic)
    for (long long ib = 0; ib < (long long)nbox; ++ib) {
        int z = (int)(ib % tp->dim[2]), y = (int)((ib / tp->dim[2]) % tp->dim[1]), xx = (int)(ib / ((size_t)tp->dim[1] * tp->dim[2]));
        int K[3] = {lo[0] + xx, lo[1] + y, lo[2] + z};
        for (int n = 0; n < nb; ++n) {
            cplx acc = {0.0, 0.0};
            for (int i2 = 0; i2 < npk; ++i2) {
                int d0 = K[0] - Gk[3 * i2] - dlo[0], d1 = K[1] - Gk[3 * i2 + 1] - dlo[1], d2 = K[2] - Gk[3 * i2 + 2] - dlo[2];
                size_t di = ((size_t)d0 * dd[1] + d1) * dd[2] + d2;
                cplx t = {th[2 * di], th[2 * di + 1]};
                acc = cadd(acc, cmul(t, ck[(size_t)(sel ? sel[n] : n) * npk + i2]));
            }
            tp->T[(size_t)n * nbox + ib] = acc;
        }
    }
    free(Kd);
    free(th);
}

/* Bounds of every K = G + G1 - G0 needed by the pairs of k. */
static void thetapsi_bounds(const OraSys *s, int ik, int *lo, int *hi) {
    for (int x = 0; x < 3; ++x) { lo[x] = 1 << 30; hi[x] = -(1 << 30); }
    for (int iq = 0; iq < n_k(s); ++iq) {
        int ikp, G0[3];
        ora_fold(s, ik, iq, &ikp, G0);
        const int *Gp = s->Gk + 3 * s->pw_off[ikp];
        const int *Ga = s->Gaux + 3 * s->gaux_off[iq];
        for (int x = 0; x < 3; ++x) {
            int amin = 1 << 30, amax = -(1 << 30), pmin = 1 << 30, pmax = -(1 << 30);
            for (int g = 0; g < s->n_ipw[iq]; ++g) { int v = Ga[3 * g + x]; if (v < amin) amin = v; if (v > amax) amax = v; }
            for (int g = 0; g < s->npw[ikp]; ++g) { int v = Gp[3 * g + x]; if (v < pmin) pmin = v; if (v > pmax) pmax = v; }
            if (s->n_ipw[iq] == 0 || s->npw[ikp] == 0) continue;
            if (amin + pmin - G0[x] < lo[x]) lo[x] = amin + pmin - G0[x];
            if (amax + pmax - G0[x] > hi[x]) hi[x] = amax + pmax - G0[x];
        }
    }
    for (int x = 0; x < 3; ++x) if (lo[x] > hi[x]) { lo[x] = 0; hi[x] = 0; }
}

/* nb: bands of the ThetaPsi table (all of k, or the selected ones) */
static void zipw_from_thetapsi(const OraSys *s, int ik, int iq, const ThetaPsi *tp, int nb, int inner, cplx *Z) {
    int ikp, G0[3];
    ora_fold(s, ik, iq, &ikp, G0);
    int no = s->n_occ[ikp];
    int npp = s->npw[ikp], ng = s->n_ipw[iq];
    const int *Gp = s->Gk + 3 * s->pw_off[ikp];
    const int *Ga = s->Gaux + 3 * s->gaux_off[iq];
    const cplx *cp = cptr(s->c, s->c_off[ikp]);
    size_t nbox = (size_t)tp->dim[0] * tp->dim[1] * tp->dim[2];
    double rs = 1.0 / sqrt(ora_omega(s));
#pragma omp parallel for schedule(dynamic) if (inner)
    for (int g = 0; g < ng; ++g)
        for (int m = 0; m < no; ++m)
            for (int n = 0; n < nb; ++n) {
                cplx acc = {0.0, 0.0};
                for (int i1 = 0; i1 < npp; ++i1) {
                    int K0 = Ga[3 * g] + Gp[3 * i1] - G0[0] - tp->lo[0];
                    int K1 = Ga[3 * g + 1] + Gp[3 * i1 + 1] - G0[1] - tp->lo[1];
                    int K2 = Ga[3 * g + 2] + Gp[3 * i1 + 2] - G0[2] - tp->lo[2];
                    size_t bi = ((size_t)K0 * tp->dim[1] + K1) * tp->dim[2] + K2;
                    acc = cadd(acc, cconjmul(cp[(size_t)m * npp + i1], tp->T[(size_t)n * nbox + bi]));
                }
                Z[((size_t)g * no + m) * nb + n] = cscale(acc, rs);
            }
}

int ora_zipw(const OraSys *s, int ik, int iq, double *Zout) {
    int lo[3], hi[3];
    thetapsi_bounds(s, ik, lo, hi);
    ThetaPsi tp;
    thetapsi_build(s, ik, lo, hi, NULL, s->n_bands[ik], &tp);
    zipw_from_thetapsi(s, ik, iq, &tp, s->n_bands[ik], 0, (cplx *)Zout);
    free(tp.T);
    return 0;
}

/* ------------------------------------------------- multipole transform */

/* Sec. III.C, unitary transformation of the MT functions of one (a, L):
 * an orthogonal P x P matrix T whose first row is mu/|mu| (the function that
 * keeps the multipole moment) and whose remaining rows span the multipole-free
 * complement.  For P = 2 this is exactly the paper's two-function formula
 * (second row (mu2, -mu1)/|mu|); for P > 2 ("generally") the complement is the
 * Householder reflection that maps mu/|mu| to e_1.  Row-major output. */
void ora_transform_T(int P, const double *mu, double *T) {
    double nrm = 0.0;
    for (int i = 0; i < P; ++i) nrm += mu[i] * mu[i];
    nrm = sqrt(nrm);
    memset(T, 0, sizeof(double) * P * P);
    if (nrm == 0.0) {
        for (int i = 0; i < P; ++i) T[i * P + i] = 1.0;
        return;
    }
    if (P == 1) { T[0] = mu[0] / nrm; return; }
    if (P == 2) {
        T[0] = mu[0] / nrm; T[1] = mu[1] / nrm;
        T[2] = mu[1] / nrm; T[3] = -mu[0] / nrm;
        return;
    }
    /* w = u + s e_1 with u = mu/|mu|, s = sign(u_1); H = I - 2 w w^T / w^T w
     * maps u to -s e_1, so T = -s H has first row u and is orthogonal. */
    double u0 = mu[0] / nrm, sg = (u0 >= 0.0) ? 1.0 : -1.0;
    double *w = (double *)malloc(sizeof(double) * P);
    double ww = 0.0;
    for (int i = 0; i < P; ++i) { w[i] = mu[i] / nrm; }
    w[0] += sg;
    for (int i = 0; i < P; ++i) ww += w[i] * w[i];
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j)
            T[i * P + j] = -sg * ((i == j ? 1.0 : 0.0) - 2.0 * w[i] * w[j] / ww);
    free(w);
}

/* ------------------------------------------------------------ V^x */

/* Full projection vector of a pair, Z[I][m][n] over the whole MPB (MT part
 * first, then the interstitial plane waves in list order). */
static void z_pair(const OraSys *s, int ik, int iq, const ThetaPsi *tp, const int *sel, int nsel, int inner, cplx *Z) {
    int ikp, G0[3];
    ora_fold(s, ik, iq, &ikp, G0);
    int nb = nsel, no = s->n_occ[ikp];
    size_t mt = (size_t)n_mt(s) * no * nb;
    zmt_core(s, ik, iq, sel, nsel, inner, (double *)Z);
    zipw_from_thetapsi(s, ik, iq, tp, nsel, inner, Z + mt);
}

/* Apply the multipole transform of every (a, L, M) to the MT rows of Z
 * (Z_t = T Z) and to v (v_t = T v T^T); the interstitial rows are unchanged. */
static void transform_pair(const OraSys *s, int n_aux, int ncol, cplx *Z, cplx *v) {
    int P = s->P, nlm = (s->Lmax + 1) * (s->Lmax + 1);
    double *T = (double *)malloc(sizeof(double) * P * P);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * P * (size_t)(ncol > n_aux ? ncol : n_aux));
    for (int a = 0; a < s->n_atoms; ++a)
        for (int L = 0; L <= s->Lmax; ++L) {
            ora_transform_T(P, s->mu + (size_t)a * (s->Lmax + 1) * P + (size_t)L * P, T);
            for (int M = -L; M <= L; ++M) {
                int base = (a * nlm + lm_idx(L, M)) * P;
                /* rows of Z */
                for (int i = 0; i < P; ++i)
                    for (int cc = 0; cc < ncol; ++cc) {
                        cplx acc = {0, 0};
                        for (int j = 0; j < P; ++j) acc = cadd(acc, cscale(Z[(size_t)(base + j) * ncol + cc], T[i * P + j]));
                        tmp[(size_t)i * ncol + cc] = acc;
                    }
                for (int i = 0; i < P; ++i) memcpy(Z + (size_t)(base + i) * ncol, tmp + (size_t)i * ncol, sizeof(cplx) * ncol);
                /* rows of v */
                for (int i = 0; i < P; ++i)
                    for (int cc = 0; cc < n_aux; ++cc) {
                        cplx acc = {0, 0};
                        for (int j = 0; j < P; ++j) acc = cadd(acc, cscale(v[(size_t)(base + j) * n_aux + cc], T[i * P + j]));
                        tmp[(size_t)i * n_aux + cc] = acc;
                    }
                for (int i = 0; i < P; ++i) memcpy(v + (size_t)(base + i) * n_aux, tmp + (size_t)i * n_aux, sizeof(cplx) * n_aux);
                /* columns of v */
                for (int r = 0; r < n_aux; ++r) {
                    cplx row[64];
                    for (int i = 0; i < P; ++i) {
                        cplx acc = {0, 0};
                        for (int j = 0; j < P; ++j) acc = cadd(acc, cscale(v[(size_t)r * n_aux + base + j], T[i * P + j]));
                        row[i] = acc;
                    }
                    for (int i = 0; i < P; ++i) v[(size_t)r * n_aux + base + i] = row[i];
                }
            }
        }
    free(T);
    free(tmp);
}

/* Eq. (div final) with e^{-beta q0^2} = beta, returned as the positive
 * bracket b such that the diagonal correction is -f_nk b:
 *   b = (pi beta)^{-1/2} erf(sqrt(beta) q0)
 *       - (4 pi / (N_k Omega)) sum_{q in mesh, G: 0 < |q+G| <= q0} e^{-beta|q+G|^2}/|q+G|^2.
 * The 4 pi turns the discrete sum into (1/2pi^2) times the BZ integral of the
 * same integrand (the paper's printed prefactor lacks it). */
double ora_vdiv(const OraSys *s) {
    double beta = s->beta;
    double q0 = sqrt(-log(beta) / beta);
    double B[9];
    recip(s, B);
    double om = ora_omega(s);
    int nk = n_k(s);
    double sum = 0.0;
    int bound[3];
    for (int i = 0; i < 3; ++i) {
        double an = sqrt(s->lattice[3 * i] * s->lattice[3 * i] + s->lattice[3 * i + 1] * s->lattice[3 * i + 1] +
                         s->lattice[3 * i + 2] * s->lattice[3 * i + 2]);
        bound[i] = (int)ceil(q0 * an / (2.0 * M_PI)) + 2;
    }
    for (int iq = 0; iq < nk; ++iq) {
        int j[3];
        mesh_j(s, iq, j);
        double qf[3] = {(double)j[0] / s->mesh[0], (double)j[1] / s->mesh[1], (double)j[2] / s->mesh[2]};
        for (int g0 = -bound[0]; g0 <= bound[0]; ++g0)
            for (int g1 = -bound[1]; g1 <= bound[1]; ++g1)
                for (int g2 = -bound[2]; g2 <= bound[2]; ++g2) {
                    double f[3] = {qf[0] + g0, qf[1] + g1, qf[2] + g2};
                    double c[3];
                    cart_of(B, f, c);
                    double q2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
                    if (q2 == 0.0 || q2 > q0 * q0) continue;
                    sum += exp(-beta * q2) / q2;
                }
    }
    return erf(sqrt(beta) * q0) / sqrt(M_PI * beta) - 4.0 * M_PI / (nk * om) * sum;
}

/* V^x_{nn'}(k) of Eq. (vec-mat-vec), with the Brillouin-zone sum read as
 * (1/N_k) sum_q:
 *   V[n][n'] = -(1/N_k) sum_q sum_{m < n_occ(k-q)} sum_{I,J}
 *                 conj(Z[I,m,n]) v_IJ(q) Z[J,m,n']
 * plus, if q0term, -delta_nn' f_nk b (Eq. div final; f_nk = 1 for
 * n < n_occ(k)).  transformed = 1 evaluates the same sum in the multipole-
 * transformed basis (Z_t = T Z, v_t = T v T^T, Sec. III.C) with dense loops.
 * Bands n, n' run over sel[0..nsel) (all bands when sel is NULL); the m sum
 * always takes every occupied band of k - q.  Output V[j][j'] complex,
 * nsel^2.  OpenMP distributes the q sum (or, on meshes with fewer q points
 * than threads, the rows inside each pair); every element is summed in the
 * same order either way, and the per-q results are added in q order. */
static int vx_core(const OraSys *s, int ik, int transformed, int q0term, const int *sel, int nsel, int nql,
                   const int *qlist, double *Vout) {
    int nk = n_k(s), nb = nsel;
    int lo[3], hi[3];
    thetapsi_bounds(s, ik, lo, hi);
    ThetaPsi tp;
    thetapsi_build(s, ik, lo, hi, sel, nsel, &tp);
    cplx *part = (cplx *)calloc((size_t)nk * nb * nb, sizeof(cplx));
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    const int nqs = qlist ? nql : nk;
    const int inner = nqs < nthr;
#pragma omp parallel for schedule(dynamic, 1) if (!inner)
    for (int iqs = 0; iqs < nqs; ++iqs) {
        const int iq = qlist ? qlist[iqs] : iqs;
        int ikp, G0[3];
        ora_fold(s, ik, iq, &ikp, G0);
        int no = s->n_occ[ikp];
        int n_aux = n_mt(s) + s->n_ipw[iq];
        int ncol = no * nb;
        cplx *Z = (cplx *)malloc(sizeof(cplx) * ((size_t)n_aux * ncol + 1));
        z_pair(s, ik, iq, &tp, sel, nsel, inner, Z);
        const cplx *vq = cptr(s->v, s->v_off[iq]);
        cplx *vw = (cplx *)vq;
        cplx *vcopy = NULL;
        if (transformed) {
            vcopy = (cplx *)malloc(sizeof(cplx) * (size_t)n_aux * n_aux);
            memcpy(vcopy, vq, sizeof(cplx) * (size_t)n_aux * n_aux);
            transform_pair(s, n_aux, ncol, Z, vcopy);
            vw = vcopy;
        }
        /* Y = v Z (each Y[I][c] summed over J in ascending order) */
        cplx *Y = (cplx *)calloc((size_t)n_aux * ncol + 1, sizeof(cplx));
#pragma omp parallel for schedule(dynamic) if (inner)
        for (int I = 0; I < n_aux; ++I)
            for (int J = 0; J < n_aux; ++J) {
                cplx vij = vw[(size_t)I * n_aux + J];
                const cplx *zr = Z + (size_t)J * ncol;
                cplx *yr = Y + (size_t)I * ncol;
                for (int cc = 0; cc < ncol; ++cc) yr[cc] = cadd(yr[cc], cmul(vij, zr[cc]));
            }
        /* P[n][n'] = sum_m sum_I conj(Z[I,m,n]) Y[I,m,n'] (m outer, I inner) */
        cplx *Pq = part + (size_t)iqs * nb * nb;
#pragma omp parallel for schedule(dynamic) if (inner)
        for (int n = 0; n < nb; ++n)
            for (int m = 0; m < no; ++m)
                for (int I = 0; I < n_aux; ++I) {
                    const cplx zc = Z[(size_t)I * ncol + (size_t)m * nb + n];
                    const cplx *yr = Y + (size_t)I * ncol + (size_t)m * nb;
                    for (int n2 = 0; n2 < nb; ++n2)
                        Pq[(size_t)n * nb + n2] = cadd(Pq[(size_t)n * nb + n2], cconjmul(zc, yr[n2]));
                }
        free(Y);
        free(Z);
        free(vcopy);
    }
    cplx *V = (cplx *)Vout;
    for (int i = 0; i < nb * nb; ++i) { V[i].re = 0.0; V[i].im = 0.0; }
    for (int iqs = 0; iqs < nqs; ++iqs)
        for (int i = 0; i < nb * nb; ++i) V[i] = cadd(V[i], part[(size_t)iqs * nb * nb + i]);
    for (int i = 0; i < nb * nb; ++i) V[i] = cscale(V[i], -1.0 / nk);
    if (q0term) {
        double b = ora_vdiv(s);
        for (int j = 0; j < nb; ++j)
            if ((sel ? sel[j] : j) < s->n_occ[ik]) V[(size_t)j * nb + j].re -= b;
    }
    free(part);
    free(tp.T);
    return 0;
}

int ora_vx(const OraSys *s, int ik, int transformed, int q0term, double *Vout) {
    return vx_core(s, ik, transformed, q0term, NULL, s->n_bands[ik], 0, NULL, Vout);
}

/* The sub-block V^x[sel][sel] of ora_vx for the bands sel[0..nsel) of k. */
int ora_vx_sub(const OraSys *s, int ik, int nsel, const int *sel, int q0term, double *Vout) {
    for (int j = 0; j < nsel; ++j)
        if (sel[j] < 0 || sel[j] >= s->n_bands[ik]) return -1;
    return vx_core(s, ik, 0, q0term, sel, nsel, 0, NULL, Vout);
}

/* The terms of q in qlist[0..nq) only (no q->0 term): -(1/N_k) sum_{q in
 * qlist} of the pair products of ora_vx_sub.  A bounded piece of the sum,
 * for timing the oracle on large workloads. */
int ora_vx_part(const OraSys *s, int ik, int nsel, const int *sel, int nq, const int *qlist, double *Vout) {
    for (int j = 0; j < nsel; ++j)
        if (sel[j] < 0 || sel[j] >= s->n_bands[ik]) return -1;
    for (int i = 0; i < nq; ++i)
        if (qlist[i] < 0 || qlist[i] >= n_k(s)) return -1;
    return vx_core(s, ik, 0, 0, sel, nsel, nq, qlist, Vout);
}

/* ------------------------------------------------ LAPW representation */

/* Eq. (APW trafo), Sec. III.A: the exchange matrix in the LAPW basis of k,
 *   V_GG' = sum_{n,n'} (S c)[G][n] V[n][n'] (c^H S)[n'][G'],
 * (S c)[G][n] = sum_G'' S[G][G''] c[n][G''] = < chi_G | phi_n >,
 * (c^H S)[n'][G'] = sum_G'' conj(c[n'][G'']) S[G''][G'] = < phi_n' | chi_G' >,
 * with S[G][G'] = < chi_G | chi_G' > the overlap matrix of the basis functions
 * of k and c[n][G] the coefficients of phi_n in them.  Inputs row-major and
 * complex: S npw x npw, c nb x npw, V nb x nb; output npw x npw.  Plain loops:
 * the two brackets first, then the double sum over n, n' per element. */
int ora_lapw_trafo(int npw, int nb, const double *Sd, const double *cd, const double *Vd, double *out) {
    const cplx *S = (const cplx *)Sd, *c = (const cplx *)cd, *V = (const cplx *)Vd;
    cplx *L = (cplx *)malloc(sizeof(cplx) * ((size_t)npw * nb + 1));   /* (S c)[G][n] */
    cplx *R = (cplx *)malloc(sizeof(cplx) * ((size_t)nb * npw + 1));   /* (c^H S)[n][G'] */
#pragma omp parallel for schedule(static)
    for (int G = 0; G < npw; ++G)
        for (int n = 0; n < nb; ++n) {
            cplx acc = {0.0, 0.0};
            for (int G2 = 0; G2 < npw; ++G2) acc = cadd(acc, cmul(S[(size_t)G * npw + G2], c[(size_t)n * npw + G2]));
            L[(size_t)G * nb + n] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int n = 0; n < nb; ++n)
        for (int G = 0; G < npw; ++G) {
            cplx acc = {0.0, 0.0};
            for (int G2 = 0; G2 < npw; ++G2) acc = cadd(acc, cconjmul(c[(size_t)n * npw + G2], S[(size_t)G2 * npw + G]));
            R[(size_t)n * npw + G] = acc;
        }
    cplx *O = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (int G = 0; G < npw; ++G)
        for (int G2 = 0; G2 < npw; ++G2) {
            cplx acc = {0.0, 0.0};
            for (int n = 0; n < nb; ++n)
                for (int n2 = 0; n2 < nb; ++n2)
                    acc = cadd(acc, cmul(cmul(L[(size_t)G * nb + n], V[(size_t)n * nb + n2]), R[(size_t)n2 * npw + G2]));
            O[(size_t)G * npw + G2] = acc;
        }
    free(L);
    free(R);
    return 0;
}

/* ------------------------------------------------ k.p term at q = 0 */

/* Appendix A: terms of the BZ integrand of Eq. (divergent part) beyond 1/q^2 at
 * q = 0, from first-order k.p perturbation theory, Eq. (first order kp
 * expansion): with the momentum matrix elements p[a][m][n] = <phi_m|d_a|phi_n>
 * (a = x, y, z) and the band energies eps[n],
 *   D[a][m][n] = <phi_m | d/dq_a Phi_n> = -i p[a][m][n] / (eps[n] - eps[m])  (m != n),
 * and D = 0 for m = n and for |eps[n] - eps[m]| < deg_tol (a degenerate pair,
 * on which first-order theory does not fix the mixing).  The spherical
 * average of the second-order term is
 *   Abar[n1][n2] = (4 pi / 3) sum_a [ sum_{n < nocc} D[a][n1][n] conj(D[a][n2][n])
 *                    - (n1, n2 < nocc) sum_m conj(D[a][m][n1]) D[a][m][n2] ],
 * and it enters the q = 0 point of the discretised BZ integral (weight
 * 4 pi / (N_k Omega) per point, 1 / (4 pi) of it for the angular average):
 *   out[n1][n2] = -Abar[n1][n2] / (N_k Omega),
 * the term added to V^x(k).  Inputs complex row-major; nk_omega = N_k Omega. */
int ora_kp_term(int nb, int nocc, const double *eps, const double *pd, double nk_omega, double deg_tol, double *out) {
    const cplx *p = (const cplx *)pd;
    cplx *D = (cplx *)malloc(sizeof(cplx) * 3 * (size_t)nb * nb + 1);
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < nb; ++m)
            for (int n = 0; n < nb; ++n) {
                cplx d = {0.0, 0.0};
                double de = eps[n] - eps[m];
                if (m != n && fabs(de) >= deg_tol) {
                    cplx pm = p[((size_t)a * nb + m) * nb + n];
                    d.re = pm.im / de;     /* -i (x + i y) / de = (y - i x) / de */
                    d.im = -pm.re / de;
                }
                D[((size_t)a * nb + m) * nb + n] = d;
            }
    cplx *O = (cplx *)out;
    for (int n1 = 0; n1 < nb; ++n1)
        for (int n2 = 0; n2 < nb; ++n2) {
            cplx acc = {0.0, 0.0};
            for (int a = 0; a < 3; ++a) {
                const cplx *Da = D + (size_t)a * nb * nb;
                for (int n = 0; n < nocc; ++n) acc = cadd(acc, cmul(Da[(size_t)n1 * nb + n], cconj(Da[(size_t)n2 * nb + n])));
                if (n1 < nocc && n2 < nocc)
                    for (int m = 0; m < nb; ++m) {
                        cplx t = cconjmul(Da[(size_t)m * nb + n1], Da[(size_t)m * nb + n2]);
                        acc.re -= t.re;
                        acc.im -= t.im;
                    }
            }
            O[(size_t)n1 * nb + n2] = cscale(acc, -(4.0 * M_PI / 3.0) / nk_omega);
        }
    free(D);
    return 0;
}

/* ------------------------------------------------- MT product basis */

/* Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix a (row-major,
 * destroyed): eigenvalues in ev, eigenvectors in the columns of V. */
static void jacobi_eig(int n, double *a, double *ev, double *V) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += a[i * n + j] * a[i * n + j];
                if (i != j) off += a[i * n + j] * a[i * n + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a[p * n + q];
                if (apq == 0.0) continue;
                double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {          /* rows p, q of a: a <- J^T a */
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - sn * akq;
                    a[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - sn * aqk;
                    a[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
}

/* The on-site Coulomb integral of two radial functions of one angular channel
 * L (Laplace expansion of 1/|r - r'| and orthonormal Y_LM):
 *   4 pi/(2L+1) int int f(r) g(r') r<^L / r>^(L+1) r^2 r'^2 dr dr',
 * as the tensor product of the grid's quadrature (the kernel's kink on r = r'
 * limits the order; the pins bound the error on fine grids). */
double ora_radial_coulomb(int n_r, const double *r, const double *w, int L, const double *f, const double *g) {
    double acc = 0.0;
    for (int i = 0; i < n_r; ++i)
        for (int j = 0; j < n_r; ++j) {
            double rl = r[i] < r[j] ? r[i] : r[j], rg = r[i] < r[j] ? r[j] : r[i];
            acc += w[i] * w[j] * r[i] * r[i] * r[j] * r[j] * f[i] * g[j] * pow(rl, L) / pow(rg, L + 1);
        }
    return 4.0 * M_PI / (2 * L + 1) * acc;
}

/* Sec. III.B: the MT functions of the mixed product basis of one atom, from
 * its LAPW radial functions u_lp (Eq. FLAPW-basis) on a radial grid r_i with
 * quadrature weights w_i for int_0^S g(r) dr.  For every L:
 *   - the products u_lp u_l'p' with lp <= l'p' and |l - l'| <= L <= l + l',
 *     each normalised (int f^2 r^2 dr = 1);
 *   - for L = 0 the spherically symmetric constant function is added first and
 *     projected out of the products;
 *   - the overlap matrix of the products is diagonalised and the eigenfunctions
 *     with eigenvalue above thr are the candidates (linear-dependence removal);
 *   - the library has a fixed count P per (a, L): the P (L = 0: P - 1 after the
 *     constant) of largest eigenvalue are kept, each normalised, the sign fixed
 *     so that its largest eigenvector component is positive (a reading).
 * Outputs: M [(Lmax+1) P][n_r] on the grid, mu [(Lmax+1) P] the multipole
 * moments int M r^(L+2) dr (Sec. III.C), R [(Lmax+1) P][n_lp][n_lp] the radial
 * integrals int M u_lp u_l'p' r^2 dr, and C [(Lmax+1)][P][P] the on-site
 * Coulomb integrals 4 pi/(2L+1) int int M_P(r) M_P'(r') r<^L / r>^(L+1) r^2 r'^2
 * dr dr' (Laplace expansion of 1/|r - r'|; tensor-product quadrature).
 * Returns 0, or -(L+1) if fewer than P functions survive for that L. */
int ora_mpb_radial(int n_r, const double *r, const double *w, const double *u, int lmax, int Lmax, int P, double thr,
                   double *Mout, double *mu, double *R, double *C) {
    const int nlp = 2 * (lmax + 1);
    int maxc = nlp * (nlp + 1) / 2 + 1;
    double *f = (double *)malloc(sizeof(double) * (size_t)maxc * n_r);
    double *O = (double *)malloc(sizeof(double) * maxc * maxc);
    double *V = (double *)malloc(sizeof(double) * maxc * maxc);
    double *ev = (double *)malloc(sizeof(double) * maxc);
    int rc = 0;
    for (int L = 0; L <= Lmax && !rc; ++L) {
        /* candidate products */
        int nc = 0;
        for (int a = 0; a < nlp; ++a)
            for (int b = a; b < nlp; ++b) {
                int la = a / 2, lb = b / 2;
                if (abs(la - lb) > L || L > la + lb) continue;
                double nrm = 0.0;
                for (int i = 0; i < n_r; ++i) {
                    double v = u[(size_t)a * n_r + i] * u[(size_t)b * n_r + i];
                    f[(size_t)nc * n_r + i] = v;
                    nrm += w[i] * r[i] * r[i] * v * v;
                }
                if (nrm <= 0.0) continue;
                for (int i = 0; i < n_r; ++i) f[(size_t)nc * n_r + i] /= sqrt(nrm);
                ++nc;
            }
        /* L = 0: the constant function, normalised, projected out of the products */
        double *cst = NULL;
        if (L == 0) {
            cst = (double *)malloc(sizeof(double) * n_r);
            double nrm = 0.0;
            for (int i = 0; i < n_r; ++i) nrm += w[i] * r[i] * r[i];
            for (int i = 0; i < n_r; ++i) cst[i] = 1.0 / sqrt(nrm);
            for (int c = 0; c < nc; ++c) {
                double d = 0.0;
                for (int i = 0; i < n_r; ++i) d += w[i] * r[i] * r[i] * cst[i] * f[(size_t)c * n_r + i];
                for (int i = 0; i < n_r; ++i) f[(size_t)c * n_r + i] -= d * cst[i];
            }
        }
        /* overlap matrix and its eigenpairs */
        for (int a = 0; a < nc; ++a)
            for (int b = 0; b < nc; ++b) {
                double o = 0.0;
                for (int i = 0; i < n_r; ++i) o += w[i] * r[i] * r[i] * f[(size_t)a * n_r + i] * f[(size_t)b * n_r + i];
                O[a * nc + b] = o;
            }
        jacobi_eig(nc, O, ev, V);
        const int want = (L == 0) ? P - 1 : P;
        /* the want largest eigenvalues above the threshold, descending */
        int *pick = (int *)malloc(sizeof(int) * (want > 0 ? want : 1));
        char *used = (char *)calloc(nc > 0 ? nc : 1, 1);
        int got = 0;
        for (int k = 0; k < want; ++k) {
            int best = -1;
            for (int c = 0; c < nc; ++c)
                if (!used[c] && ev[c] > thr && (best < 0 || ev[c] > ev[best])) best = c;
            if (best < 0) break;
            used[best] = 1;
            pick[got++] = best;
        }
        if (got < want) rc = -(L + 1);
        for (int P_ = 0; P_ < P && !rc; ++P_) {
            double *M = Mout + ((size_t)L * P + P_) * n_r;
            if (L == 0 && P_ == 0) {
                memcpy(M, cst, sizeof(double) * n_r);
            } else {
                int e = pick[L == 0 ? P_ - 1 : P_];
                int big = 0;
                for (int c = 1; c < nc; ++c)
                    if (fabs(V[c * nc + e]) > fabs(V[big * nc + e])) big = c;
                double sg = V[big * nc + e] >= 0 ? 1.0 : -1.0, sc = sg / sqrt(ev[e]);
                for (int i = 0; i < n_r; ++i) {
                    double acc = 0.0;
                    for (int c = 0; c < nc; ++c) acc += V[c * nc + e] * f[(size_t)c * n_r + i];
                    M[i] = sc * acc;
                }
            }
        }
        free(pick);
        free(used);
        free(cst);
        if (rc) break;
        /* multipole moments, radial integrals, on-site Coulomb */
        for (int P_ = 0; P_ < P; ++P_) {
            const double *M = Mout + ((size_t)L * P + P_) * n_r;
            double m = 0.0;
            for (int i = 0; i < n_r; ++i) m += w[i] * M[i] * pow(r[i], L + 2);
            mu[L * P + P_] = m;
            for (int a = 0; a < nlp; ++a)
                for (int b = 0; b < nlp; ++b) {
                    double acc = 0.0;
                    for (int i = 0; i < n_r; ++i) acc += w[i] * r[i] * r[i] * M[i] * u[(size_t)a * n_r + i] * u[(size_t)b * n_r + i];
                    R[(((size_t)L * P + P_) * nlp + a) * nlp + b] = acc;
                }
            for (int Q = 0; Q < P; ++Q)
                C[((size_t)L * P + P_) * P + Q] = ora_radial_coulomb(n_r, r, w, L, M, Mout + ((size_t)L * P + Q) * n_r);
        }
    }
    free(f); free(O); free(V); free(ev);
    return rc;
}

/* ------------------------------------------------- inversion symmetry */

/* Sec. III.D: the partner of every atom under r -> -r, i.e. the atom a' whose
 * fractional position is -R_a up to integers, with the same sphere radius;
 * -1 where there is none.  Returns the number of atoms without a partner. */
int ora_inv_partner(const OraSys *s, int *partner) {
    int missing = 0;
    for (int a = 0; a < s->n_atoms; ++a) {
        partner[a] = -1;
        for (int b = 0; b < s->n_atoms && partner[a] < 0; ++b) {
            int ok = fabs(s->rmt[a] - s->rmt[b]) < 1e-12;
            for (int x = 0; x < 3 && ok; ++x) {
                double d = s->pos_frac[3 * a + x] + s->pos_frac[3 * b + x];
                ok = fabs(d - floor(d + 0.5)) < 1e-8;
            }
            if (ok) partner[a] = b;
        }
        if (partner[a] < 0) ++missing;
    }
    return missing;
}

/* Sec. III.D, Eqs. (sym MT functions) and the M = 0 rule after them: the
 * symmetrized MT functions M' as columns of S over the original Bloch MT
 * functions, M'_J = sum_I S[I][J] M_I (row-major, N_aux x N_aux complex, the
 * identity on the interstitial plane waves).  With a' the partner of a and
 * s = (-1)^(L+M):
 *   M'_(a,L,M,P)    = [M_(a,L,M,P) + s M_(a',L,-M,P)] / sqrt 2
 *   M'_(a',L,-M,P)  = i [M_(a,L,M,P) - s M_(a',L,-M,P)] / sqrt 2
 * for every M when a < a' (the reading of which atom of a pair plays "a"),
 * and for M < 0 when a' = a; for a' = a and M = 0 the function is kept for
 * even L and multiplied by i for odd L.  Returns -1 if an atom has no partner. */
int ora_sym_matrix(const OraSys *s, int n_aux, double *Sout) {
    int *partner = (int *)malloc(sizeof(int) * (s->n_atoms > 0 ? s->n_atoms : 1));
    if (ora_inv_partner(s, partner)) { free(partner); return -1; }
    cplx *S = (cplx *)Sout;
    memset(S, 0, sizeof(cplx) * (size_t)n_aux * n_aux);
    const int P = s->P, nlm = (s->Lmax + 1) * (s->Lmax + 1), nmt = n_mt(s);
    const double h = 1.0 / sqrt(2.0);
    for (int I = nmt; I < n_aux; ++I) S[(size_t)I * n_aux + I].re = 1.0;
    for (int a = 0; a < s->n_atoms; ++a) {
        const int b = partner[a];
        for (int L = 0; L <= s->Lmax; ++L)
            for (int M = -L; M <= L; ++M) {
                const double sg = ((L + M) % 2 == 0) ? 1.0 : -1.0;
                for (int p = 0; p < P; ++p) {
                    const int A = (a * nlm + lm_idx(L, M)) * P + p;       /* M_(a,L,M,P) */
                    const int B = (b * nlm + lm_idx(L, -M)) * P + p;      /* M_(a',L,-M,P) */
                    if (a == b && M == 0) {
                        if (L % 2 == 0) S[(size_t)A * n_aux + A].re = 1.0;
                        else S[(size_t)A * n_aux + A].im = 1.0;
                        continue;
                    }
                    if (!(a < b || (a == b && M < 0))) continue;       /* handled with its pair */
                    /* column A: the first function of the pair, column B: the second */
                    S[(size_t)A * n_aux + A].re = h;
                    S[(size_t)B * n_aux + A].re = sg * h;
                    S[(size_t)A * n_aux + B].im = h;
                    S[(size_t)B * n_aux + B].im = -sg * h;
                }
            }
    }
    free(partner);
    return 0;
}

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
