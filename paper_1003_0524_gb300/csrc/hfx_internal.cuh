// hfx_internal.cuh -- context layout, device helpers and kernel declarations of
// the exchange-matrix library (sm_103a).  Nothing here is part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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
    std::vector<int> G;          // host copy (for boxes)
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
    __nv_bfloat16 *d_Ap = nullptr;  // unused (the slices of every q live in hfx_ctx::s_ap)
};

struct Scratch {                 // growable device buffers
    void *p = nullptr;
    size_t bytes = 0;
};

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
    double *d_R = nullptr;       // [n_atoms][(Lmax+1)P][nlp][nlp]
    double *d_mu = nullptr;      // [n_atoms][(Lmax+1)P]
    double *d_T = nullptr;       // [n_atoms][Lmax+1][P][P] multipole transforms
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
    std::shared_ptr<void> zipw_plan;
};

namespace hfx {

// ------------------------------------------------------------ host helpers
int set_err(hfx_ctx *ctx, int code, const std::string &msg);
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
// embedding [[Vr,-Vi],[Vi,Vr]] of VD.
void launch_build_ap(const double2 *d_VD, __nv_bfloat16 *d_Ap, int *d_aexp, int D, int naux, int N0, int N0pad,
                     int Dpad, int RS, cudaStream_t st);
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
// The channel blocks of Y (rows [0, N0)).  With d_VD non-null (the double-FP32
// kernel, block_y_couples(P, N0)) it also adds to each channel's mu != 0 row
// N0 + ch its couplings to the channel's mu = 0 functions, v_t[N0+ch, mu=0 of ch]
// Z[mu=0 of ch]: the only nonzeros of the dense-block rows in the mu = 0 columns,
// which gemm1 then skips (launch it after gemm1).
template <typename V>
void launch_block_y(const QDesc *d_q, int nq, const double2 *const *d_VB, const double2 *const *d_VD, const V *d_Z,
                    double2 *d_Y, long long RSc, int P, int N0, long long maxcols, cudaStream_t st);
bool block_y_couples(int P, int N0);
// skip_mu0: leave out the mu = 0 columns of v_t's dense-block rows (added by launch_block_y)
int launch_gemm1_tc(hfx_ctx *ctx, const __nv_bfloat16 *d_Ap_all, long long ap_rows, const int *d_aexp, const QDesc *h_q,
                    const QDesc *d_q, int nq, const __nv_bfloat16 *d_ZS, const int *d_zexp, double2 *d_Y, long long RSc,
                    long long NC, int N0, int N0pad, int Dpad, int RS, bool skip_mu0, void *d_tiles_buf, size_t tiles_cap);
int launch_gemm2_tc(hfx_ctx *ctx, const __nv_bfloat16 *d_ZS, const __nv_bfloat16 *d_YS, const int *d_zexp,
                    const int *d_yexp, long long NC, int RS, int HS, int N0pad, const PairDesc *h_pairs,
                    const PairDesc *d_pairs, int npairs, const QDesc *d_q, int NB, const long long *d_praw_off,
                    double *d_praw, void *d_tiles_buf, size_t tiles_cap);

// ------------------------------------------------------------ interstitial projections on the tensor cores (k_zipw_tc.cu)
struct ZipwTcInput {
    std::vector<int> kset, qs;              // k points with pairs; q of the batch
    std::vector<PairDesc> pairs;            // host copy of the batch pairs
    const PairDesc *d_pairs;
    const double2 *const *d_ck;             // per k: c [nb][npw]
    const int *const *d_Gk;                 // per k: G [npw][3]
    const int *d_npw, *d_nb;
    const double2 *const *d_Tk;             // per k: T_n(K) [nb][box] (FP64)
    int nb_max;
    int tlo[3], tdim[3];                    // T box
    double2 *d_Z;                           // projections [col][RSc]
    long long RSc;
    cudaEvent_t ev_gemm0 = nullptr, ev_gemm1 = nullptr;   // recorded around the GEMM launch if set
};
int zipw_tc_prepare_and_launch(hfx_ctx *ctx, const ZipwTcInput &in);

// ------------------------------------------------------------ stage-1 products on the tensor cores (k_cgemm_tc.cu)
// T_n(K) of every k of kset (Sec. III.B), written to d_T + toff[k] + n * box.
int thetapsi_tc(hfx_ctx *ctx, const std::vector<int> &kset, const double2 *d_theta, const int dlo[3], const int ddim[3],
                const int tlo[3], const int tdim[3], double2 *d_T, const std::vector<size_t> &toff);
struct ZmtTcState {                         // operand slices of Z^MT, valid for one build
    bool ready = false;
    int Kh = 0, npairs_a = 0, npairs_pad = 0;
    long long RA = 0, RB = 0;
    std::vector<long long> blk_row0, blk_rows;   // [k][a]
    std::vector<int> kbase, pk, pm;              // (k', m) pair list of every atom block
    std::vector<std::pair<int, int>> blocks;     // (k, a) of the A blocks
    size_t oA = 0, oB = 0, oae = 0, obe = 0, oro = 0, opk = 0, fixed_bytes = 0;
};
int zmt_tc_prepare(hfx_ctx *ctx, ZmtTcState &zs, const std::vector<int> &kset, const std::vector<double2 *> &hB,
                   long long RSc, int N0, int sparse);
// Z^MT of the pairs of one batch (Sec. III.A) into d_Z; d_tables: device scratch for per-batch tables.
int zmt_tc_launch(hfx_ctx *ctx, const ZmtTcState &zs, const std::vector<PairDesc> &pairs, long long RSc, double2 *d_Z,
                  void *d_tables, size_t tables_cap);

// ------------------------------------------------------------ kernels (finish, k_finish.cu)
void launch_reduce_pairs(const PairDesc *d_pairs, const int *d_kstart, const int *d_klist_pairs, int nk_in_batch,
                         const int *d_klist, const double *d_praw, const long long *d_praw_off, int NB, int raw_format,
                         double2 *const *d_vacc, const int *d_nb_k, int nb_max, cudaStream_t st);
void launch_finish(double2 *const *d_vacc, double2 *const *d_V, const int *d_nb_k, const int *d_no_k, int nk,
                   int nb_max, double inv_nk, double q0b, int q0_on, double *d_Ex, cudaStream_t st);

}  // namespace hfx
