/*
 * hfx.h -- C ABI of the GB300 (sm_103a) library that builds the nonlocal
 * Hartree-Fock exchange matrix of the PBE0-in-FLAPW method (Betzinger,
 * Friedrich, Bluegel; Sec. III):
 *
 *   V^x_{nn'}(k) = -(1/N_k) sum_q sum_{m<n_occ(k-q)} sum_{IJ}
 *                   conj(Z_q[I,m,n]) v_IJ(q) Z_q[J,m,n']           Eq. (vec-mat-vec)
 *                 - delta_nn' f_nk b                               Eq. (div final)
 *
 * with the mixed-product-basis projections Z_q[I,m,n] = < M_I^q phi_{m,k-q} | phi_{n,k} >
 * (Sec. III.B) and the Coulomb matrix v(q) of Eq. (coulomb matrix), which the
 * library makes block-sparse with the multipole transformation of Sec. III.C.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Status: every function returns HFX_OK (0) or a negative HFX_E* code; no
 *   exception, abort or exit crosses the ABI.  hfx_strerror() names a code and
 *   hfx_last_error() returns the context's last message (valid until the next
 *   call on that context).
 * - Ownership: inputs are deep-copied (to the device) before the call
 *   returns; the caller keeps and may free its buffers.  Outputs go into
 *   caller-allocated buffers of the documented size.
 * - Complex numbers are interleaved double pairs (C99 double _Complex layout).
 *   Matrices are row-major, dense, 0-based.
 * - Index conventions (Eq. FLAPW-basis and Sec. III.B):
 *     LAPW MT index  lmp = 2*(l*l + l + m) + p,  p in {0,1},  N_lmp = 2(lmax+1)^2
 *     radial index   lp  = 2*l + p
 *     MPB MT index   I   = (a*(Lmax+1)^2 + L*L + L + M)*P + Pidx   (atom outermost)
 *     MPB IPW index  I   = N_MT + g, g over the per-q plane-wave list,
 *                    N_MT = n_atoms (Lmax+1)^2 P,  N_aux(q) = N_MT + n_ipw(q)
 *     k mesh         k = sum_i (j_i/N_i) b_i,  ik = (j0*N1 + j1)*N2 + j2 (Gamma-centred);
 *                    the q mesh is the same set and k - q is folded back into it.
 * - One context is not thread-safe.  All device work runs on the stream given
 *   in hfx_options (NULL = the legacy default stream) on the device given there.
 * - A context keeps every input resident in device memory; building V^x leaves
 *   the result on the device until hfx_get_exchange copies it out.
 */
#ifndef HFX_H
#define HFX_H

#include <stddef.h>

#if defined(__GNUC__)
#define HFX_API __attribute__((visibility("default")))
#else
#define HFX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status */
#define HFX_OK 0
#define HFX_EINVAL (-1)        /* bad size, index, pointer or option */
#define HFX_ENOTHERM (-2)      /* v(q) not Hermitian within tolerance */
#define HFX_ENONFINITE (-3)    /* NaN or Inf in an input */
#define HFX_EMISSING (-4)      /* build requested before every required set_* call */
#define HFX_EDEVICE (-5)       /* CUDA error (message in hfx_last_error) */
#define HFX_ETIMEOUT (-6)      /* a bounded device wait expired */
#define HFX_ENOMEM (-7)        /* host or device allocation failed */
#define HFX_ENOTSPARSE (-8)    /* sparse mode forced but v(q) is not block-sparse */
#define HFX_EUNSUPPORTED (-9)  /* size or option outside what this build supports */

/* -------------------------------------------------------------- types */
typedef struct hfx_ctx hfx_ctx;

/* Crystal and basis description (Eq. FLAPW-basis, Sec. III.B). */
typedef struct {
    double lattice[9];        /* rows a_1, a_2, a_3 in bohr */
    int n_atoms;              /* atoms (MT spheres) per cell, >= 1 */
    const double *pos_frac;   /* [n_atoms][3] fractional positions */
    const double *rmt;        /* [n_atoms] MT radii S_a (bohr), >= 0, non-overlapping */
    int lmax;                 /* LAPW angular cutoff (0..8) */
    int Lmax;                 /* MPB angular cutoff (0..8), Sec. III.B */
    int n_rad;                /* P: MT product functions per (atom, L) after the
                                 linear-dependence removal (1..16) */
    int mesh[3];              /* k mesh N_1 x N_2 x N_3, each >= 1 */
} hfx_system;

enum {
    HFX_PREC_FP64 = 0,        /* every step in FP64 on the CUDA cores (the plain FP64 GPU build) */
    HFX_PREC_SLICED = 1       /* contractions on the tensor cores in exact fixed-point
                                 BF16 slice arithmetic (four 8-bit slices per operand
                                 line, exact class sums, compensated combination);
                                 projections, transform, q->0 term and q sum in FP64 */
};
enum {
    HFX_SPARSE_AUTO = 0,      /* use the block-sparse form if every v(q) has it */
    HFX_SPARSE_ON = 1,        /* require it (HFX_ENOTSPARSE otherwise) */
    HFX_SPARSE_OFF = 2        /* dense vector-matrix-vector products */
};

typedef struct {
    int precision;            /* HFX_PREC_* */
    int sparse;               /* HFX_SPARSE_* */
    int q0_term;              /* nonzero: add Eq. (div final) to the occupied diagonal */
    double beta;              /* Eq. (F(q)) parameter, > 0; q0 from e^{-beta q0^2} = beta */
    double herm_tol;          /* relative Hermiticity tolerance for v(q) */
    double sparse_tol;        /* relative size of elements treated as zero in the
                                 transformed v(q) */
    void *stream;             /* cudaStream_t (NULL: legacy default stream) */
    int device;               /* CUDA device ordinal */
    size_t work_bytes;        /* device budget for the working buffers of one batch of
                                 (k, q) pairs (0: what the device has free after the
                                 per-build buffers); a batch holds whole pairs, so the
                                 k points of one q may be split over several batches */
    int use_graph;            /* nonzero: the first build of a plan is captured as one
                                 CUDA graph (on a private stream) and later builds with
                                 the same inputs structure replay it on `stream` */
    int tile_nb_zhy;          /* band block of the Z^H Y tiles: 8..64, multiple of 8
                                 (0: least padded work) */
    int tile_nb_zipw;         /* band block of the interstitial tiles: 8..64, multiple
                                 of 8 (0: fewest padded bands up to 40) */
    int kp_term;              /* nonzero: add the k.p term at q = 0 of Appendix A to V^x
                                 (needs hfx_set_momentum for every k) */
    double kp_deg_tol;        /* energy difference (Ha) below which two bands count as
                                 degenerate and their k.p mixing is left out */
    int test_fail_wait;       /* fault-injection hook for tests: nonzero makes the next
                                 build's Z^H Y kernel wait on a barrier that nothing
                                 completes; the bounded wait expires after about 1 ms,
                                 the kernel drains its copies and MMAs, frees its TMEM
                                 and returns, and the build returns HFX_ETIMEOUT.  The
                                 flag clears itself after that build. */
    int inversion;            /* nonzero: the system has inversion symmetry and is given
                                 in the real-valued form of Sec. III.D (see "Inversion
                                 symmetry" below); V^x is real symmetric and the
                                 contractions run on real operands */
} hfx_options;

/* Inversion symmetry (Sec. III.D), hfx_options.inversion != 0
 * ------------------------------------------------------------
 * Every atom a has a partner a' (possibly a itself) with R_a' = -R_a + T_a,
 * T_a a lattice vector, the same sphere radius (checked at hfx_create:
 * HFX_EINVAL), and the same radial integrals and multipole moments (checked at
 * the build: HFX_EINVAL).  The wave functions obey phi(-r) = phi(r)^*, which
 * with the conventions of hfx_set_kpoint reads
 *     c_G(n,k) real,    A^{a'}_{l,-m,p}(n,k) = (-1)^(l+m) e^{i k.T_a} conj(A^a_{l,m,p}(n,k))
 * (checked by hfx_set_kpoint within herm_tol: HFX_EINVAL).  The Coulomb matrix
 * is given over the symmetrized MT functions of Eqs. (sym MT functions), which
 * keep the labels (a, L, M, P) of the index convention above:
 *     M'_(a,L,M,P)   = [M_(a,L,M,P) + s M_(a',L,-M,P)] / sqrt 2,     s = (-1)^(L+M)
 *     M'_(a',L,-M,P) = i [M_(a,L,M,P) - s M_(a',L,-M,P)] / sqrt 2
 * for every M when a < a', for M < 0 when a' = a, and M'_(a,L,0,P) = M or i M
 * (L even or odd) when a' = a; the interstitial plane waves are unchanged.  In
 * that basis v(q) is real symmetric (imaginary parts beyond herm_tol:
 * HFX_EINVAL).  V^x is returned as before, with zero imaginary parts.  The
 * library packs two occupied bands m, m+1 of k - q into one complex column
 * (Z' real per band, so Z'_m + i Z'_{m+1} carries both and Re(Z^H v Z) sums
 * their contributions), which halves the columns of every contraction; the
 * Coulomb apply then runs on the real operand alone.  hfx_set_products and
 * hfx_get_products are not available in this mode (HFX_EUNSUPPORTED). */

/* Layout of the Coulomb matrix passed to hfx_set_coulomb. */
enum {
    HFX_LAYOUT_DENSE = 0,       /* v(q) in the MPB order above (Eq. coulomb matrix) */
    HFX_LAYOUT_TRANSFORMED = 1, /* v_t = T v T^T in the same index positions, T the
                                   multipole transform of hfx_get_transform (Sec. III.C):
                                   MT function P' = 0 of every (a, L, M) is the one with
                                   a multipole, P' >= 1 are multipole-free */
    HFX_LAYOUT_TRANSFORMED_ONSITE = 2 /* as TRANSFORMED, but the rows and columns of the
                                   multipole-free functions (P' >= 1) are ignored: the
                                   library fills them at the build with the on-site
                                   blocks T C T^T of hfx_set_radial_functions (every
                                   atom needs it) and zero elsewhere, which is exact:
                                   a multipole-free function makes no potential outside
                                   its sphere (Sec. III.C, Fig. 1) */
};

/* Per-build statistics (filled if the pointer is non-NULL). */
typedef struct {
    double ms_total;          /* device time of the build (CUDA events) */
    double ms_stage1;         /* projections Z (MT + interstitial) */
    double ms_contract;       /* Coulomb apply and Z^H (vZ) */
    double ms_finish;         /* q sum, q->0 term, E_x */
    double useful_flops;      /* the method's flop count (Sec. III.C sparse form) */
    int n_pairs;              /* (k, q) pairs processed */
    int n_batches;            /* q batches */
    int sparse_used;          /* 1 if the block-sparse form was used */
    int n_launches;           /* kernels launched by this build */
    double ms_zipw;           /* interstitial projection kernel (all launches; the GEMM
                                 kernel alone in the sliced build) */
    double ms_apply;          /* Coulomb apply Y = v_t Z (dense block, all launches) */
    double ms_zhy;            /* Z^H Y contraction (all launches) */
    double flops_apply;       /* useful flops of the dense-block apply: 8 D^2 per column */
    double flops_zhy;         /* useful flops of Z^H Y: 8 N_aux n per column */
    double flops_zipw;        /* useful flops of the interstitial projection */
    int graph_replayed;       /* 1 if the build was the replay of a captured CUDA graph */
    int tile_nb_zhy;          /* band block of the Z^H Y tiles used */
    int tile_nb_zipw;         /* band block of the interstitial tiles used (0: FP64 build) */
    double flops_apply_exec;  /* flops of the dense-block apply as executed: the sliced
                                 build applies the upper triangle U of v_t (half
                                 diagonal) and adds P' + P'^H, 8 D (D+1)/2 per column;
                                 the FP64 build applies all of v_t, 8 D^2 */
} hfx_stats;

/* ------------------------------------------------------------ entry points */

/* Fill *opt with defaults: SLICED, sparse AUTO, q0 term on, beta = 0.005
 * (Sec. III.E), herm_tol 1e-10, sparse_tol 1e-12, NULL stream, device 0. */
HFX_API void hfx_default_options(hfx_options *opt);

/* Create a context for one spin channel.  Validates the system (sizes,
 * finite values, non-overlapping spheres), selects the device, and builds the
 * Gaunt table G(LM; lm; l'm') = int Y*_LM Y*_lm Y_l'm' (MT product functions,
 * Sec. III.B) on the device.  *out receives the context (NULL on failure). */
HFX_API int hfx_create(const hfx_system *sys, const hfx_options *opt, hfx_ctx **out);

/* Radial data of one atom (Sec. III.B-C).
 *   R  [(Lmax+1)*P][2(lmax+1)][2(lmax+1)] real: radial product integrals
 *      int_0^S M_{aLP}(r) u_{lp}(r) u_{l'p'}(r) r^2 dr, symmetric in lp <-> l'p'
 *      (checked, HFX_EINVAL).
 *   mu [(Lmax+1)*P] real: multipole moments mu_{aLP} = int_0^S M_{aLP} r^{L+2} dr,
 *      which define the unitary transform of Sec. III.C. */
HFX_API int hfx_set_radial(hfx_ctx *ctx, int atom, const double *R, const double *mu);

/* The MT product functions of one atom built from its LAPW radial functions
 * (Sec. III.B), on the GPU in FP64, replacing the inputs of hfx_set_radial:
 *   n_r, r, w  radial grid: r [n_r] increasing in (0, R_MT], w [n_r] quadrature
 *              weights of int_0^R_MT g(r) dr (2 <= n_r <= 8192)
 *   u          [2(lmax+1)][n_r] u_lp(r) on the grid, lp = 2l + p (Eq. FLAPW-basis)
 *   threshold  eigenvalue threshold of the linear-dependence removal (the paper
 *              uses 1e-4), > 0
 * For every L the products u_lp u_l'p' (lp <= l'p', |l - l'| <= L <= l + l') are
 * normalised, for L = 0 the constant function is added and projected out of them,
 * the overlap matrix of the products is diagonalised, and the P eigenfunctions of
 * largest eigenvalue above the threshold (P - 1 for L = 0) become M_aLP,
 * normalised, each with its largest eigenvector component positive.  From them
 * the library computes the multipole moments mu_aLP = int M r^(L+2) dr
 * (Sec. III.C), the radial integrals R = int M u_lp u_l'p' r^2 dr, and the on-site
 * Coulomb blocks C_aL[P][P'] = 4 pi/(2L+1) int int M_P M_P' r<^L/r>^(L+1) r^2 r'^2
 * (Eq. coulomb matrix restricted to one sphere; used by
 * HFX_LAYOUT_TRANSFORMED_ONSITE).  Errors: HFX_EINVAL (grid, pointer, or fewer
 * than P functions above the threshold for some L), HFX_ENONFINITE. */
HFX_API int hfx_set_radial_functions(hfx_ctx *ctx, int atom, int n_r, const double *r, const double *w,
                                     const double *u, double threshold);

/* The basis built by hfx_set_radial_functions for one atom; any pointer may be NULL:
 *   M [(Lmax+1) P][n_r], mu [(Lmax+1) P], R [(Lmax+1) P][2(lmax+1)][2(lmax+1)],
 *   C [Lmax+1][P][P].  HFX_EMISSING if the atom has none. */
HFX_API int hfx_get_radial_basis(hfx_ctx *ctx, int atom, double *M, double *mu, double *R, double *C);

/* Wave functions of one k point (Eq. FLAPW-basis), uploaded to the device.
 *   n_bands   band window n_max of Sec. III (V^x is n_bands x n_bands), >= 1
 *   n_occ     occupied bands (f_nk = 1 for n < n_occ), 0..n_bands
 *   npw, G    [npw][3] integer reciprocal vectors of the plane waves |k+G| <= Gmax
 *   c         [n_bands][npw] complex: interstitial coefficients, phi = Omega^{-1/2} sum c e^{i(k+G)r}
 *   A         [n_bands][n_atoms][N_lmp] complex: MT coefficients of phi in the home cell */
HFX_API int hfx_set_kpoint(hfx_ctx *ctx, int ik, int n_bands, int n_occ, int npw, const int *G,
                   const double *c, const double *A);

/* Coulomb matrix of one q point (Eq. coulomb matrix), built once per SCF cycle.
 *   n_ipw, G_aux  [n_ipw][3] integer G of the interstitial plane waves M^q_G
 *   v             N_aux x N_aux complex, row-major with row stride ld (complex
 *                 elements, ld >= N_aux); Hermitian (HFX_ENOTHERM beyond
 *                 herm_tol); v(q=0) is the finite part v'(0) of Eq. (div + nondiv part)
 *   layout        HFX_LAYOUT_DENSE: v in the MPB order above; the library applies
 *                 the multipole transform v_t = T v T^T in FP64 on the device at
 *                 the next build (after every hfx_set_radial).
 *                 HFX_LAYOUT_TRANSFORMED: v is already v_t (Sec. III.C, Fig. 1) for
 *                 the T of hfx_get_transform; it is used as given.
 * Errors: HFX_EINVAL (index, size, ld or layout), HFX_ENONFINITE, HFX_ENOTHERM. */
HFX_API int hfx_set_coulomb(hfx_ctx *ctx, int iq, int n_ipw, const int *G_aux, const double *v, int ld, int layout);

/* The multipole transform T_aL of one atom and L (Sec. III.C), P x P real,
 * row-major: row 0 is mu_aL / |mu_aL| (the function with a multipole), rows
 * 1..P-1 an orthonormal basis of the multipole-free functions (Gram-Schmidt
 * on the unit vectors, in order).  Requires hfx_set_radial for the atom. */
HFX_API int hfx_get_transform(hfx_ctx *ctx, int atom, int L, double *T);

/* Supply the projection vectors of one (k, q) pair directly instead of
 * computing them from the wave functions (Eq. vec-mat-vec):
 *   Z  [N_aux(q)][n_occ(k-q)][n_bands(k)] complex, MPB order above.
 * Z == NULL removes an earlier override.  The override persists across builds. */
HFX_API int hfx_set_products(hfx_ctx *ctx, int ik, int iq, const double *Z);

/* Copy the projection vectors of one pair, as computed by the last build,
 * into Z (layout of hfx_set_products; untransformed MPB order).  Requires a
 * preceding build with keep_products = 1 (see hfx_build_all). */
HFX_API int hfx_get_products(hfx_ctx *ctx, int ik, int iq, double *Z);

/* Build V^x(k) for every k of the mesh and E_x, leaving them on the device.
 * keep_products != 0 also keeps every pair's Z for hfx_get_products (memory
 * permitting, else HFX_ENOMEM).  Requires hfx_set_radial for every atom,
 * hfx_set_kpoint for every k and hfx_set_coulomb for every q (HFX_EMISSING). */
HFX_API int hfx_build_all(hfx_ctx *ctx, int keep_products, hfx_stats *st);

/* Build V^x for one k only (its N_k pairs) and copy it to Vx
 * [n_bands][n_bands] complex. */
HFX_API int hfx_build_exchange(hfx_ctx *ctx, int ik, double *Vx, hfx_stats *st);

/* Copy V^x(k) of the last hfx_build_all into Vx [n_bands][n_bands] complex. */
HFX_API int hfx_get_exchange(hfx_ctx *ctx, int ik, double *Vx);

/* Device pointer of V^x(k) of the last build ([n_bands][n_bands] complex
 * double, valid until the next build or hfx_destroy). */
HFX_API int hfx_exchange_device_ptr(hfx_ctx *ctx, int ik, const double **Vx_dev);

/* Exchange energy of one spin channel of the last build (Eq. HF exchange
 * energy): E_x = (1/2)(1/N_k) sum_k sum_{n<n_occ(k)} Re V^x_nn(k). */
HFX_API int hfx_get_energy(hfx_ctx *ctx, double *Ex);

/* The q->0 bracket b of Eq. (div final) (FP64, computed on the device):
 * b = (pi beta)^{-1/2} erf(sqrt(beta) q0)
 *     - (4 pi / (N_k Omega)) sum_{q, G: 0<|q+G|<=q0} e^{-beta|q+G|^2}/|q+G|^2. */
HFX_API int hfx_get_q0_bracket(hfx_ctx *ctx, double *b);

/* Allocation-free q->0 bracket (no counterpart in the paper: an interface
 * choice of this library).  Writes the same value as hfx_get_q0_bracket, but
 * needs no context and allocates no device memory, for callers that cannot
 * allocate at that point: processes whose device memory is entirely owned by
 * another allocator (for example a framework's caching pool), and code that
 * must avoid the device-wide synchronisation that cudaMalloc/cudaFree may
 * perform.
 *   lattice      [9] rows a_i (bohr)
 *   mesh         [3] k mesh, each 1..64
 *   beta         the decay parameter of the auxiliary function, in (0, 1);
 *                q0 follows from e^{-beta q0^2} = beta
 *   bracket_dev  DEVICE pointer to one double owned by the caller; written
 *                asynchronously on `stream`
 *   stream       cudaStream_t (NULL: legacy default stream), current device
 * The partial sums of the reduction live in a fixed 512 KiB device array
 * inside the library (65536 doubles): each GPU on which the library is used
 * holds its own copy until the process exits.  Sizes needing more partial
 * sums than that (k points x (2 ceil(q0 |a_1| / 2 pi) + 5) > 65536) return
 * HFX_EUNSUPPORTED.  Every call looks up the array's address on the current
 * device (cudaGetSymbolAddress, which allocates nothing; the first call on a
 * device also loads the library's module there, so make that first call
 * before any stream capture).  Calls that overlap on the same device (for
 * example on two streams) race on that device's array and must be ordered by
 * the caller; calls on different devices use separate copies.  Every partial
 * sum is written before it is read, so nothing needs clearing between calls.
 * Errors: HFX_EINVAL (bad pointer, mesh or beta), HFX_ENONFINITE,
 * HFX_EUNSUPPORTED, HFX_EDEVICE (no device or launch failure). */
HFX_API int hfx_q0_bracket_noalloc(const double *lattice, const int *mesh, double beta, double *bracket_dev,
                                   void *stream);

/* Inputs of the k.p term at q = 0 (Appendix A, Eq. first order kp expansion)
 * for the bands of k:
 *   eps  [n_bands] band energies (Ha)
 *   p    [3][n_bands][n_bands] complex momentum matrix elements
 *        <phi_m| d/dr_a |phi_n> (a = x, y, z), anti-Hermitian in (m, n) (checked
 *        against herm_tol, HFX_EINVAL).
 * With opt.kp_term the build adds to V^x(k) the term -Abar/(N_k Omega): Abar is
 * the spherical average of the second-order terms of the integrand of
 * Eq. (divergent part), from D_mn = -i p_mn / (eps_n - eps_m) (pairs closer than
 * kp_deg_tol left out), for occupied (n1, n2)
 *   (4 pi/3) sum_a [sum_{n occ} D_n1n conj(D_n2n) - sum_m conj(D_mn1) D_mn2],
 * otherwise (4 pi/3) sum_a sum_{n occ} D_n1n conj(D_n2n).  Requires hfx_set_kpoint(k). */
HFX_API int hfx_set_momentum(hfx_ctx *ctx, int ik, const double *eps, const double *p);

/* Overlap matrix S_GG'(k) = <chi_G|chi_G'> of the LAPW basis functions of k
 * (Eq. APW Hamiltonian, Sec. III.A), npw x npw complex, Hermitian (checked,
 * HFX_ENOTHERM), rows in the order of the plane-wave list given to
 * hfx_set_kpoint, row stride ld >= npw.  Requires hfx_set_kpoint(k). */
HFX_API int hfx_set_overlap(hfx_ctx *ctx, int ik, const double *S, int ld);

/* The exchange matrix in the LAPW basis of every k (Eq. APW trafo):
 *   V_GG'(k) = sum_{n,n'} (S c)[G][n] V^x_nn'(k) (c^H S)[n'][G'],
 * with c the coefficients of hfx_set_kpoint and V^x of the last hfx_build_all,
 * in FP64 on the device (three batched complex GEMMs over all k).  Requires a
 * complete build and hfx_set_overlap for every k (HFX_EMISSING).  st->ms_total
 * and st->useful_flops describe the transform. */
HFX_API int hfx_lapw_transform_all(hfx_ctx *ctx, hfx_stats *st);

/* Copy V_GG'(k) of the last hfx_lapw_transform_all into Vgg (npw x npw
 * complex, row stride ld >= npw). */
HFX_API int hfx_get_lapw_exchange(hfx_ctx *ctx, int ik, double *Vgg, int ld);

/* Release every host and device resource of the context (NULL is a no-op). */
HFX_API void hfx_destroy(hfx_ctx *ctx);

/* Static description of a status code. */
HFX_API const char *hfx_strerror(int code);

/* Last error message of the context ("" if none). */
HFX_API const char *hfx_last_error(const hfx_ctx *ctx);

/* Library version string. */
HFX_API const char *hfx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HFX_H */
