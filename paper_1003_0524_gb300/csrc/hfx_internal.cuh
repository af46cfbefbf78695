// hfx_internal.cuh -- context layout, device helpers and kernel declarations of
// the exchange-matrix library (sm_103a).  Nothing here is part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hfx.h"

namespace hfx {

// ------------------------------------------------------------ limits
constexpr int kMaxL = 8;            // lmax, Lmax
constexpr int kMaxP = 16;           // radial functions per (a, L)
constexpr int kMaxAtoms = 4096;
constexpr int kMaxBandsTile = 64;   // n-block of the tensor-core Z^H Y tile

// Device error word values (hfx_ctx::d_err)
enum DevErr : int { kDevOk = 0, kDevTimeoutTma = 1, kDevTimeoutMma = 2, kDevTimeoutEpi = 3, kDevBadIndex = 4 };

// ------------------------------------------------------------ complex helpers
template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename V> __host__ __device__ __forceinline__ V cmk(decltype(V().x) re, decltype(V().x) im) {
    V r; r.x = re; r.y = im; return r;
}
template <typename V> __host__ __device__ __forceinline__ V cfma(V a, V b, V acc) {       // acc + a*b
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
template <typename V> __host__ __device__ __forceinline__ V cfma_conj(V a, V b, V acc) {  // acc + conj(a)*b
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}

// ------------------------------------------------------------ batch layout
// One q batch: the column space of every q is the list of (k, m, n) with
// col = colbase + kbase[k] + m * nb[k] + n; the row space is the permuted MPB
// [mu=0 MT functions (N0) | dense block D = mu!=0 MT functions + IPW].
struct PairDesc {           // one (k, q) pair of a batch (device copy)
    int ik, iq, ikp;        // k, q, k' = k - q folded
    int g0[3];              // G0 = k - q - k'
    int nb, no;             // n_bands(k), n_occ(k')
    long long col0;         // first column of the pair in the batch column space
    int qslot;              // index of q inside the batch
    int pad;
};

struct QDesc {              // one q of a batch (device copy)
    int iq;
    int nipw;
    int naux;               // N_MT + nipw
    int D;                  // dense-block size
    long long colbase;      // first column of q
    long long ncols;        // columns of q
    int pair0, npairs;      // pairs of q in the batch pair list
};

// ------------------------------------------------------------ context
struct KPoint {
    int nb = 0, no = 0, npw = 0;
    bool set = false;
    int *d_G = nullptr;          // [npw][3]
    double2 *d_c = nullptr;      // [nb][npw]
    double2 *d_A = nullptr;      // [nb][n_atoms][N_lmp]
    // the occupied bands in their role m of k - q: d_c, d_A and no themselves,
    // or with inversion symmetry (Sec. III.D) the packed pairs
    // X_j = X_{2j} - i X_{2j+1} (own buffers), nom = ceil(no / 2)
    double2 *d_cm = nullptr;     // [nom][npw]
    double2 *d_Am = nullptr;     // [nom][n_atoms][N_lmp]
    int nom = 0;
    std::vector<int> G;          // host copy (for boxes)
    // inputs of the k.p term at q = 0 (Appendix A) and its result
    double *d_eps = nullptr;     // [nb]
    double2 *d_p = nullptr;      // [3][nb][nb]
    double2 *d_kp = nullptr;     // [nb][nb]  term added to V^x
    int kp_nb = 0;               // band count the buffers were made for
    bool kp_set = false;
};

struct QPoint {
    int nipw = 0;
    bool set = false;
    int *d_G = nullptr;          // [nipw][3]
    double2 *d_v = nullptr;      // [naux][naux] original order
    std::vector<int> G;
    // derived (after the transform): dense-block rows of v_t, all columns
    double2 *d_VD = nullptr;     // [D][naux]   permuted order
    double2 *d_VB = nullptr;     // [n_ch][P-1][P]  mu=0 rows inside their channel
    size_t vd_cap = 0, vb_cap = 0;  // allocated elements of d_VD, d_VB
    int layout = HFX_LAYOUT_DENSE;  // how v was given (dense, or already transformed)
};

struct Scratch {                 // growable device buffers
    void *p = nullptr;
    size_t bytes = 0;
};

// Host-side image of device tables: every put() starts at a 256-byte boundary
// and returns its offset; the image is uploaded once and the offsets resolve
// against the device copy.
struct HostArena {
    std::vector<unsigned char> buf;
    size_t put(const void *src, size_t bytes) {
        size_t o = (buf.size() + 255) / 256 * 256;
        buf.resize(o + (bytes ? bytes : 1), 0);
        if (bytes) std::memcpy(buf.data() + o, src, bytes);
        return o;
    }
    template <typename T> size_t put(const std::vector<T> &v) { return put(v.data(), v.size() * sizeof(T)); }
};

// Offsets of 256-byte aligned sub-buffers of one device allocation.
struct Layout {
    size_t off = 0;
    size_t place(size_t bytes) {
        size_t o = off;
        off = (off + bytes + 255) / 256 * 256;
        return o;
    }
};

struct BuildPlan;   // hfx_api.cu

}  // namespace hfx

struct hfx_ctx {
    hfx_system sys;
    std::vector<double> pos, rmt;
    hfx_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;

    int nk = 0, nlm = 0, nLM = 0, nlmp = 0, nlp = 0, P = 0, nch = 0, nmt = 0;
    double omega = 0.0, B[9] = {0};

    std::vector<hfx::KPoint> kp;
    std::vector<hfx::QPoint> qp;
    std::vector<char> rset;
    std::vector<int> partner;    // inversion partner of every atom (inversion mode)
    std::vector<double> hR, hmu; // host copies of the radial inputs (partner checks)
    // the MT product basis built from radial functions (hfx_set_radial_functions)
    std::vector<std::vector<double>> rad_M;   // per atom [(Lmax+1) P][n_r]
    std::vector<int> rad_nr;
    std::vector<double> rad_C;                // [n_atoms][Lmax+1][P][P] on-site Coulomb blocks
    std::vector<char> rad_set;
    bool rad_C_dirty = false;
    double *d_radC = nullptr;                 // device copy of rad_C
    double *d_R = nullptr;       // [n_atoms][(Lmax+1)P][nlp][nlp]
    double *d_mu = nullptr;      // [n_atoms][(Lmax+1)P]
    double *d_T = nullptr;       // [n_atoms][Lmax+1][P][P] multipole transforms
    double *d_Tid = nullptr;     // the same shape, identity blocks (v given already transformed)
    bool T_valid = false;        // d_T matches the current multipoles
    double *d_gaunt = nullptr;   // [nLM][nlm][lmax+1]
    double *d_posf = nullptr;    // [n_atoms][3]
    int *d_err = nullptr;        // device error word

    bool coulomb_dirty = true;   // transform must be redone
    bool sparse_used = false;
    int N0 = 0;                  // mu=0 rows (sparse) or 0 (dense)
    double q0_bracket = 0.0;
    bool q0_valid = false;

    // overrides of the projection vectors, original order
    std::map<std::pair<int, int>, double2 *> zover;

    // outputs of the last build
    std::vector<double2 *> d_V;  // per k [nb][nb]
    std::vector<int> V_nb;       // allocated size of d_V[k]
    double *d_Ex = nullptr;
    bool built = false;

    // kept projections (original order, FP64), keyed by pair
    std::map<std::pair<int, int>, double2 *> zkeep;

    // scratch
    hfx::Scratch s_theta, s_thpsi, s_B, s_zc, s_zs, s_ys, s_y64, s_praw, s_vacc, s_pairs, s_qd,
        s_misc, s_ap, s_aexp, s_xexp, s_zipw, s_cgT, s_cgZ;

    // bumped whenever a plane-wave list, an aux list or a band window changes;
    // host tables built from the structure are reused while it stays the same
    uint64_t struct_epoch = 0;
    // the cached build plan (device tables, scratch layout, captured graph)
    std::shared_ptr<hfx::BuildPlan> plan;

    // the LAPW representation (Eq. APW trafo): overlaps per k, results of the last transform
    std::vector<double2 *> d_S;
    std::vector<int> S_npw;
    hfx::Scratch s_lapw, s_lapw_tab;
    std::vector<size_t> lapw_off;
    bool lapw_valid = false;
};

namespace hfx {

// ------------------------------------------------------------ host helpers
int set_err(hfx_ctx *ctx, int code, const std::string &msg);
// Record a timing event (an event node of the graph while the stream captures).
void record_event(cudaEvent_t e, cudaStream_t st);
// k' = k - q folded into the mesh and G0 = k - q - k'
void fold_kq(const hfx_ctx *ctx, int ik, int iq, int *ikp, int *g0);
// Build V^x(k) for every k of kset (hfx_plan.cu): plan cache, graph capture, execution.
int build_run(hfx_ctx *ctx, const std::vector<int> &kset, int keep, hfx_stats *st);
// Drop the cached plan and every build buffer.
void plan_release(hfx_ctx *ctx);
int cuda_check(hfx_ctx *ctx, cudaError_t e, const char *what);
int scratch_reserve(hfx_ctx *ctx, Scratch &s, size_t bytes);

// ------------------------------------------------------------ kernels (setup, k_setup.cu)
// Gaunt table G[LM][lm][l2] = int Y*_LM Y*_lm Y_{l2, m+M} by Gauss-Legendre
// quadrature of associated Legendre functions.
void launch_gaunt(double *d_gaunt, int Lmax, int lmax, cudaStream_t st);
// Multipole transforms T_{aL} (Sec. III.C), FP64.
void launch_transform_T(const double *d_mu, double *d_T, int n_atoms, int Lmax, int P, cudaStream_t st);
// Step-function Fourier coefficients on an integer box (FP64).
void launch_theta(double2 *d_theta, const int lo[3], const int dim[3], const double *B, double omega,
                  const double *d_posf, const double *d_rmt, int n_atoms, cudaStream_t st);
// v_t = T v T^T, permuted into the dense-block rows (VD) and the mu=0 blocks (VB);
// off-pattern magnitude is max-reduced into *d_offmax, |v_t| into *d_absmax.
void launch_transform_v(const double2 *d_v, double2 *d_VD, double2 *d_VB, const double *d_T, int n_atoms,
                        int Lmax, int P, int nipw, int sparse, unsigned long long *d_offmax,
                        unsigned long long *d_absmax, cudaStream_t st);
// Fixed-point slices (four BF16 planes, per-row exponents) of the real
// embedding [[Ur,-Ui],[Ui,Ur]] of U, the dense-block rows of the upper triangle
// of v_t with half its diagonal; interleave: the real and imaginary rows of each
// row of U adjacent (complex path), else in two blocks (real path).
void launch_build_ap(const double2 *d_VD, __nv_bfloat16 *d_Ap, int *d_aexp, int D, int naux, int N0, int N0pad,
                     int Dpad, int RS, int interleave, cudaStream_t st);
// q->0 bracket of Eq. (div final) into *d_out (FP64); d_partial holds
// q0_partial_count() doubles.
void launch_q0_bracket_impl(double *d_out, double *d_partial, const int mesh[3], const double *B, double omega,
                            double beta, const double *lattice, cudaStream_t st);
size_t q0_partial_count(const int mesh[3], double beta, const double *lattice);

// ------------------------------------------------------------ kernels (stage 1, k_stage1.cu)
template <typename R>
void launch_thetapsi(const double2 *d_theta, const int dlo[3], const int ddim[3], const int tlo[3],
                     const int tdim[3], const double2 *d_c, const int *d_G, int nb, int npw,
                     typename C2<R>::T *d_out, cudaStream_t st);
template <typename R>
void launch_bmat(const double2 *d_A, const double *d_R, const double *d_T, const double *d_gaunt,
                 int n_atoms, int lmax, int Lmax, int P, int nb, int use_T, typename C2<R>::T *d_B,
                 cudaStream_t st);
template <typename R>
void launch_zmt(const PairDesc *d_pairs, int npairs, const QDesc *d_q, typename C2<R>::T *const *d_Bk,
                const double2 *const *d_Ak, const double *d_posf, const int mesh[3], int n_atoms, int nLM, int P,
                int nlmp, int N0, int sparse, int no_max, typename C2<R>::T *d_Z, long long RSc, cudaStream_t st);
template <typename R>
int launch_zipw(const PairDesc *d_pairs, const int *d_kpairs, int nk, int nb_max, const QDesc *d_q, int nq,
                typename C2<R>::T *const *d_Tk, const int tlo[3], const int tdim[3], const double2 *const *d_ck,
                const int *const *d_Gk, const int *d_npw, int npw_max, const int *const *d_Gaux, const int *d_nb_k,
                double omega, int rowbase_ipw, typename C2<R>::T *d_Z, long long RSc, cudaStream_t st);
template <typename R>
void launch_override(const double2 *d_user, const PairDesc &pr, int naux, const double *d_T, int n_atoms, int Lmax,
                     int P, int N0, int sparse, typename C2<R>::T *d_Z, long long RSc, int nmt, cudaStream_t st);
// Sec. III.C: the mu = 0 rows and columns of v_t (transformed index positions)
// from the on-site Coulomb blocks C [n_atoms][Lmax+1][P][P] of the radial basis.
void launch_onsite_fill(double2 *d_v, int naux, const double *d_C, const double *d_T, int n_atoms, int Lmax, int P,
                        cudaStream_t st);
// Sec. III.D: Z' = S^H Z on the MT rows of every column of a batch, with the
// row operations of sym_row_ops (pairs of rows and lone rows).
struct SymOp { int r1, r2, kind, pad; };   // kind 0: pair s = +1, 1: pair s = -1, 2: lone row times -i
std::vector<SymOp> sym_row_ops(const hfx_ctx *ctx, int N0, int sparse);
template <typename V>
void launch_sym_rows(V *d_Z, long long RSc, long long ncols, const SymOp *d_ops, int nops, cudaStream_t st);
template <typename R>
void launch_unpermute(const typename C2<R>::T *d_Z, const PairDesc &pr, int naux, const double *d_T, int n_atoms,
                      int Lmax, int P, int N0, int sparse, long long RSc, int nmt, double2 *d_out, cudaStream_t st);

// ------------------------------------------------------------ kernels (FP64 contraction, k_contract64.cu)
struct ZGemmBatch {         // C = op(A) * B, complex double, K = K1 * K2
    const double2 *A, *B;
    double2 *C;
    int M, N, K1, K2;
    long long sAi, sAk2, sAk1, sBk2, sBk1, sBj, sCi, sCj;
    int conjA;
};
void launch_zgemm64(const ZGemmBatch *d_b, int nbatch, int maxM, int maxN, cudaStream_t st);
void launch_block64(const QDesc *d_q, int nq, const double2 *const *d_VB, const double2 *d_Z, double2 *d_Y,
                    long long RSc, int nch, int P, int N0, long long maxcols, cudaStream_t st);

// ------------------------------------------------------------ kernels (tensor-core contraction, k_contract_tc.cu)
template <typename V>
void launch_slice_cols(const V *d_Z, long long RSc, const QDesc *d_q, int nq, long long NC, long long maxcols, int N0,
                       int N0pad, int Dpad, int RS, __nv_bfloat16 *d_XS, int *d_exp, cudaStream_t st);
// The channel blocks of Y' = U Z (rows [0, N0)), U the upper triangle of v_t
// with half its diagonal.  (With d_VD non-null, the double-FP32 kernel would
// also add the dense rows' couplings to the mu = 0 functions, the lower
// triangle; the Hermitian split passes null.)
template <typename V>
void launch_block_y(const QDesc *d_q, int nq, const double2 *const *d_VB, const double2 *const *d_VD, const V *d_Z,
                    double2 *d_Y, long long RSc, int P, int N0, long long maxcols, cudaStream_t st);
bool block_y_couples(int P, int N0);
// GEMM1 tiles of one batch (host) and its launch: Y' = U Z for the dense-block
// rows, U the upper triangle of v_t with half its diagonal (the slices of
// launch_build_ap), K of every row tile from its first row on.
// real_v: v_t is real (inversion symmetry), so the real rows of Y' need only the
// real half of K and the imaginary rows only the imaginary half.
int gemm1_tiles(const QDesc *h_q, int nq, int N0pad, bool real_v, std::vector<unsigned char> &out);
int launch_gemm1_tc(hfx_ctx *ctx, const __nv_bfloat16 *d_Ap_all, long long ap_rows, const int *d_aexp, const QDesc *d_q,
                    const __nv_bfloat16 *d_ZS, const int *d_zexp, double2 *d_Y, long long RSc, long long NC, int N0,
                    int N0pad, int Dpad, int RS, const void *d_tiles, int ntiles);
// real_form: the Z^H Y tiles of the inversion-symmetric path (only Re P', two
// row blocks per tile; band blocks of 16, 32, 48 or 64, see gemm2_real_form)
int gemm2_tiles(const PairDesc *h_pairs, int npairs, int NB, bool real_form, std::vector<unsigned char> &out);
int gemm2_check_nb(int NB);
bool gemm2_real_form(int NB);
int launch_gemm2_tc(hfx_ctx *ctx, const __nv_bfloat16 *d_ZS, const __nv_bfloat16 *d_YS, const int *d_zexp,
                    const int *d_yexp, long long NC, int RS, int HS, int N0pad, const PairDesc *d_pairs, const QDesc *d_q,
                    int NB, const long long *d_praw_off, double *d_praw, const void *d_tiles, int ntiles,
                    int fail_wait, bool real_form);

// ------------------------------------------------------------ interstitial projections on the tensor cores (k_zipw_tc.cu)
struct ZipwBuild {                          // per build: rows (k', m), segment grid, C slices
    bool ok = false;
    int R = 0, Rpad = 0, nmtile = 0, nL = 0, gx0 = 0, gy0 = 0, By = 0, nsegp_max = 0, Kp = 0;
    int NBt = 0, nblk = 0, nbpad = 0, nzb = 0, nb_max = 0;
    int tlo[3] = {0, 0, 0}, tdim[3] = {0, 0, 0};
    int sx0 = 0, sx1 = 0, sy0 = 0, sy1 = 0, sz0 = 0, sz1 = 0;   // extent of the segment starts
    std::vector<int> rowbase;               // first row of every k'
    size_t o_rowk = 0, o_rowm = 0, o_line = 0, o_sst = 0, o_sz0 = 0, o_seg = 0, o_nch = 0, o_runs = 0, o_kall = 0;
    size_t s_a = 0, s_aexp = 0, s_eT = 0, scratch_bytes = 0, a_elems = 0;
    size_t tq_bytes_per_slot = 0;           // sliced T of one k (all copies, planes, bands)
};
struct ZipwBatch {                          // per batch: shifts, tiles, aux lookup
    bool ok = false;
    int ntiles = 0, nslot = 0;
    int amin[3] = {0, 0, 0}, ad[3] = {1, 1, 1};
    size_t o_gtab = 0, o_pinfo = 0, o_w = 0, o_tiles = 0, o_kslot = 0;
    size_t tq_bytes = 0;
};
int zipw_tc_valid_nb(int nb);
int zipw_tc_plan_build(hfx_ctx *ctx, const std::vector<int> &kset, int nb_max, const int tlo[3], const int tdim[3],
                       int nb_tile, HostArena &tab, ZipwBuild &zb);
int zipw_tc_plan_batch(hfx_ctx *ctx, const ZipwBuild &zb, const std::vector<int> &qs, const std::vector<PairDesc> &pairs,
                       HostArena &tab, ZipwBatch &bt);
int zipw_tc_run_build(hfx_ctx *ctx, const ZipwBuild &zb, const char *dtab, char *dscr, const double2 *const *d_ck,
                      const int *const *d_Gk, const int *d_npw, const double2 *const *d_Tk, const int *d_nb);
// The interstitial rows come out G-major into d_ZI [g][NCi] (the kernel's
// stores then fill whole sectors) and are transposed into d_Z after the kernel.
int zipw_tc_run_batch(hfx_ctx *ctx, const ZipwBuild &zb, const ZipwBatch &bt, const char *dtab, const char *dscr,
                      __nv_bfloat16 *dTq, const PairDesc *d_pairs, const double2 *const *d_Tk, const int *d_nb,
                      double2 *d_Z, long long RSc, double2 *d_ZI, long long NCi, const QDesc *d_qd, int nq,
                      long long maxcols, int max_nipw, cudaEvent_t ev0, cudaEvent_t ev1, int *nlaunch);

// ------------------------------------------------------------ stage-1 products on the tensor cores (k_cgemm_tc.cu)
struct TpPlan {                             // T_n(K) of every k of the build (Sec. III.B)
    bool ok = false;
    int NU = 0, Kh = 0, npairs = 0, ntiles = 0;
    long long RA = 0, RB = 0;
    size_t o_uo = 0, o_ui = 0, o_uio = 0, o_rk = 0, o_rn = 0, o_co = 0, o_ro = 0, o_ti = 0, o_hc = 0, o_np = 0;
    size_t s_A = 0, s_B = 0, s_ae = 0, s_be = 0, scratch_bytes = 0;
};
int thetapsi_tc_plan(hfx_ctx *ctx, const std::vector<int> &kset, const int ddim[3], const int tdim[3],
                     const std::vector<size_t> &toff, HostArena &tab, TpPlan &tp);
int thetapsi_tc_run(hfx_ctx *ctx, const TpPlan &tp, const char *dtab, char *dscr, const double2 *d_theta, const int dlo[3],
                    const int ddim[3], const int tlo[3], const int tdim[3], double2 *d_T, int *nlaunch);
struct ZmtPlan {                            // operand slices of Z^MT, per build
    bool ok = false;
    int Kh = 0, npairs_a = 0, npairs_pad = 0, nblocks = 0;
    long long RA = 0, RB = 0, maxrows = 0;
    std::vector<long long> blk_row0, blk_rows;   // [k][a]
    std::vector<int> kbase;                      // first (k', m) pair of every k'
    std::vector<std::pair<int, int>> blocks;     // (k, a) of the A blocks
    size_t o_ro = 0, o_pk = 0, o_bk = 0, o_ba = 0, o_br = 0, o_nb = 0, o_hb = 0, o_ha = 0, o_pk2 = 0, o_pm = 0, o_br0 = 0;
    size_t s_A = 0, s_B = 0, s_ae = 0, s_be = 0, scratch_bytes = 0;
};
struct ZmtBatch {
    bool ok = false;
    int ntiles = 0;
    size_t o_co = 0, o_ph = 0, o_ti = 0;
};
int zmt_tc_plan(hfx_ctx *ctx, const std::vector<int> &kset, const std::vector<double2 *> &hB, long long RSc, int N0,
                int sparse, HostArena &tab, ZmtPlan &zs);
int zmt_tc_run_prepare(hfx_ctx *ctx, const ZmtPlan &zs, const char *dtab, char *dscr, int *nlaunch);
int zmt_tc_plan_batch(hfx_ctx *ctx, const ZmtPlan &zs, const std::vector<PairDesc> &pairs, long long RSc, HostArena &tab,
                      ZmtBatch &zb);
int zmt_tc_run_batch(hfx_ctx *ctx, const ZmtPlan &zs, const ZmtBatch &zb, const char *dtab, char *dscr, double2 *d_Z,
                     int *nlaunch);

// ------------------------------------------------------------ kernels (finish, k_finish.cu)
void launch_reduce_pairs(const PairDesc *d_pairs, const int *d_kstart, const int *d_klist_pairs, int nk_in_batch,
                         const int *d_klist, const double *d_praw, const long long *d_praw_off, int NB, int raw_format,
                         int real_part, double2 *const *d_vacc, const int *d_nb_k, int nb_max, cudaStream_t st);
// V = -(1/N_k) Vacc - q->0 term (+ the k.p term d_kp[k] if d_kp is non-null), and E_x.
void launch_finish(double2 *const *d_vacc, double2 *const *d_V, const int *d_nb_k, const int *d_no_k, int nk,
                   int nb_max, double inv_nk, double q0b, int q0_on, double2 *const *d_kp, double *d_Ex,
                   cudaStream_t st);
// The k.p term at q = 0 (Appendix A) of every k: -Abar / (N_k Omega) into d_kp[k].
void launch_kp_term(const double *const *d_eps, const double2 *const *d_p, double2 *const *d_kp, const int *d_nb_k,
                    const int *d_no_k, int nk, int nb_max, double nk_omega, double deg_tol, cudaStream_t st);

}  // namespace hfx
