// k_contract_tc.cu -- the contraction on the 5th-generation tensor cores
// (tcgen05.mma kind::f16 with BF16 operands, FP32 accumulators in TMEM,
// operands staged by TMA into swizzled shared memory), in
// fixed-point slice arithmetic that makes every tensor-core sum exact.
//
// Slices.  Every operand line (a row of A, a column of B) shares one power of
// two 2^e with e chosen so that the line's largest magnitude is below 2^e.  An
// element x is cut into four 8-bit integer slices,
//   x = 2^e (s0 2^-8 + s1 2^-16 + s2 2^-24 + s3 2^-32) + r,  |s0| <= 256, |s1..3| <= 128,
// each stored exactly as a BF16 number.  A product of two lines is the sum of
// the ten slice products s_i t_j with i + j <= 3, grouped by weight class
// w = i + j (weight 2^-8(w+2)).  Every class is accumulated in its own TMEM
// accumulator; since all summands are integers and a class sum over at most
// 256 K elements stays below 2^24, the FP32 accumulation is exact whatever
// the rounding mode of the tensor-core adder.  After each K group of <= 256
// the four class sums are combined, scaled by 2^(e_A + e_B) and added into
// compensated FP32 (hi, lo) pairs on the CUDA cores.  The result carries about
// 2^-33 relative error per element line, far below what the exchange matrix
// needs, with no systematic bias.
//
// Complex arithmetic uses the real embedding [[Re, -Im], [Im, Re]].
//   GEMM1 (per q, all k of the batch):  Y_D = v_t[D, D] Z_D          (Fig. 1 dense block; the mu = 0
//        columns of these rows hold only each channel's couplings, added with the channel blocks)
//   GEMM2 (per pair (k,q)):             P = sum_m Z_m^H Y_m          (Eq. vec-mat-vec)
// The q sum is then done in FP64 (k_finish.cu).
//
// Every wait is bounded (about two seconds); on expiry the kernel records an
// error code, stops issuing work, lets its in-flight copies and MMAs drain
// (again bounded), frees its TMEM and returns.
#include <algorithm>
#include <type_traits>
#include <string>

#include "tc_ptx.cuh"

namespace hfx {

using namespace tc;

namespace {

// ------------------------------------------------------------- column slicing
// For every column of the batch: exponent over its rows (real and imaginary
// parts of rows [0, N0) and [N0, N0 + D_q) of Zc), then slices into
// XS[p][col][u]: u in [0, HS) real parts, [HS, 2 HS) imaginary parts (mu=0
// rows padded to N0pad, dense rows padded to Dpad).  One warp per column; in
// the slicing pass each lane takes four consecutive rows, so every plane is
// written with 8-byte stores (N0pad and HS are multiples of 64).
__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <typename V>
__global__ void __launch_bounds__(256, 4) slice_cols_kernel(const V *__restrict__ Z, long long RSc, const QDesc *__restrict__ qd, int N0,
                                  int N0pad, int Dpad, int RS, long long NC, __nv_bfloat16 *__restrict__ XS,
                                  int *__restrict__ xexp) {
    const QDesc q = qd[blockIdx.y];
    const int HS = N0pad + Dpad;
    const int wpb = blockDim.x / 32, lane = threadIdx.x % 32;
    const long long plane = NC * RS;
    for (long long c = (long long)blockIdx.x * wpb + threadIdx.x / 32; c < q.ncols; c += (long long)gridDim.x * wpb) {
        const long long col = q.colbase + c;
        const V *z = Z + col * RSc;
        const int nrow = N0 + q.D;
        unsigned long long mx = 0;
        for (int r = lane; r < nrow; r += 32) {
            V v = z[r];
            mx = max(mx, max(abs_bits((double)v.x), abs_bits((double)v.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const int e = line_exp_bits(mx);
        if (lane == 0) xexp[col] = e;
        const long long base = col * RS;
        for (int u0 = 4 * lane; u0 < HS; u0 += 128) {
            // the four rows u0..u0+3 lie in one region (N0pad is a multiple of 64)
            int row0, nvalid;
            if (u0 < N0pad) { row0 = u0; nvalid = N0 - u0; }
            else { row0 = N0 + (u0 - N0pad); nvalid = q.D - (u0 - N0pad); }
            __nv_bfloat16 sr[4][NPL], si[4][NPL];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                double xr = 0.0, xi = 0.0;
                if (t < nvalid) {
                    V v = z[row0 + t];
                    xr = (double)v.x;
                    xi = (double)v.y;
                }
                slice4(xr, e, sr[t]);
                slice4(xi, e, si[t]);
            }
#pragma unroll
            for (int p = 0; p < NPL; ++p) {
                uint2 wr = make_uint2(pack_bf16x2(sr[0][p], sr[1][p]), pack_bf16x2(sr[2][p], sr[3][p]));
                uint2 wi = make_uint2(pack_bf16x2(si[0][p], si[1][p]), pack_bf16x2(si[2][p], si[3][p]));
                *reinterpret_cast<uint2 *>(XS + p * plane + base + u0) = wr;
                *reinterpret_cast<uint2 *>(XS + p * plane + base + HS + u0) = wi;
            }
        }
    }
}

// Weight of v_B[ch, i, s] in U, the upper triangle of v_t with half its
// diagonal, in the order [mu=0 | mu!=0 | IPW]: s = 0 is the coupling of mu = 0
// function i to the channel's mu != 0 function (a dense-block column, above the
// diagonal); s >= 1 is mu = 0 function s - 1 of the same channel.
__device__ __forceinline__ double upper_weight(int i, int s) {
    return s == 0 ? 1.0 : (s - 1 > i ? 1.0 : (s - 1 == i ? 0.5 : 0.0));
}

// Y rows of the mu=0 functions (on-site blocks of Fig. 1), FP64, with the
// upper part U of the blocks.
template <typename V>
__global__ void block_y_kernel(const QDesc *__restrict__ qd, const double2 *const *__restrict__ VB,
                               const V *__restrict__ Z, double2 *__restrict__ Y, long long RSc, int P, int N0) {
    const QDesc q = qd[blockIdx.y];
    const double2 *vb = VB[blockIdx.y];
    long long total = q.ncols * N0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int u = (int)(e % N0);
        long long col = q.colbase + e / N0;
        int ch = u / (P - 1), i = u % (P - 1);
        const V *z = Z + col * RSc;
        const double2 *row = vb + ((size_t)ch * (P - 1) + i) * P;
        V z0 = z[N0 + ch];
        double2 acc = cmul(row[0], make_double2((double)z0.x, (double)z0.y));
        for (int s = 1; s < P; ++s) {
            V zs = z[ch * (P - 1) + s - 1];
            const double w = upper_weight(i, s);
            acc = cfma(make_double2(w * row[s].x, w * row[s].y), make_double2((double)zs.x, (double)zs.y), acc);
        }
        Y[col * RSc + u] = acc;
    }
}

// x = hi + lo to within 2^-47 |x|, hi and lo FP32, from the bits of x with
// integer operations (no FP64 conversion): hi keeps the sign, the exponent and
// the top 23 stored mantissa bits (truncated), lo the remaining 29 bits (the
// integer conversion rounds them to 24).  For |x| < 2^-74 (and zero) lo = 0,
// for |x| < 2^-126 hi = 0 as well; |x| must stay below 2^128.
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
    const uint32_t sg = bh & 0x80000000u;
    const int e = (int)((bh >> 20) & 0x7ffu);
    const bool nh = e >= 897, nl = e >= 949;
    hi = __uint_as_float(nh ? sg | ((uint32_t)(e - 896) << 23) | ((bh & 0xfffffu) << 3) | (bl >> 29) : sg);
    const float r = __uint2float_rn(bl & 0x1fffffffu);                   // the 29 low bits, as an integer
    lo = nl ? __uint_as_float(__float_as_uint(r * __uint_as_float((uint32_t)(e - 948) << 23)) | sg) : 0.0f;
}

// Y rows of the mu = 0 functions (on-site blocks of Fig. 1) with the upper
// part U of v_t: for channel ch,
// Y[ch (P-1) + i] = v_B[ch, i, 0] Z[N0 + ch] + sum_{s >= 1} w(i, s) v_B[ch, i, s] Z[ch (P-1) + s - 1],
// w = upper_weight.  One thread per (column, channel) computes its P - 1 rows
// in double-FP32 arithmetic (about 2^-44 relative; the rows are sliced to
// 2^-32 of the column maximum next), so the kernel runs on the FP32 units
// rather than GB300's narrow FP64 pipe.  The blocks of q are split into shared
// memory once.
template <int P>
__global__ void block_y_df_kernel(const QDesc *__restrict__ qd, const double2 *const *__restrict__ VB,
                                  const double2 *const *__restrict__ VD, const double2 *__restrict__ Z,
                                  double2 *__restrict__ Y, long long RSc, int N0) {
    extern __shared__ float4 vbs[];   // [N0 * P] blocks, then [N0] couplings: (hi re, lo re, hi im, lo im)
    const QDesc q = qd[blockIdx.y];
    const double2 *vb = VB[blockIdx.y];
    const int nch = N0 / (P - 1);
    for (int i = threadIdx.x; i < N0 * P; i += blockDim.x) {
        const double w = upper_weight((i / P) % (P - 1), i % P);
        const double2 v = vb[i];
        float4 f;
        split_f64(w * v.x, f.x, f.y);
        split_f64(w * v.y, f.z, f.w);
        vbs[i] = f;
    }
    float4 *vcs = vbs + N0 * P;   // v_t[N0 + ch, ch (P-1) + i]: row ch of the dense block
    if (VD) {
        const double2 *vd = VD[blockIdx.y];
        for (int i = threadIdx.x; i < N0; i += blockDim.x) {
            const int ch = i / (P - 1);
            const double2 v = vd[(size_t)ch * q.naux + i];
            float4 f;
            split_f64(v.x, f.x, f.y);
            split_f64(v.y, f.z, f.w);
            vcs[i] = f;
        }
    }
    __syncthreads();
    const long long total = q.ncols * nch;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(e % nch);
        const long long col = q.colbase + e / nch;
        const double2 *z = Z + col * RSc;
        float zrh[P], zrl[P], zih[P], zil[P];
#pragma unroll
        for (int s = 0; s < P; ++s) {
            const double2 v = z[s == 0 ? N0 + ch : ch * (P - 1) + s - 1];
            split_f64(v.x, zrh[s], zrl[s]);
            split_f64(v.y, zih[s], zil[s]);
        }
#pragma unroll
        for (int i = 0; i < P - 1; ++i) {
            const float4 *row = vbs + (size_t)(ch * (P - 1) + i) * P;
            float Sr = 0.f, Er = 0.f, Si = 0.f, Ei = 0.f;
#pragma unroll
            for (int s = 0; s < P; ++s) {
                const float4 v = row[s];
                df_mac(v.x, v.y, zrh[s], zrl[s], Sr, Er);
                df_mac(-v.z, -v.w, zih[s], zil[s], Sr, Er);
                df_mac(v.x, v.y, zih[s], zil[s], Si, Ei);
                df_mac(v.z, v.w, zrh[s], zrl[s], Si, Ei);
            }
            Y[col * RSc + ch * (P - 1) + i] = make_double2(f32pair_to_f64(Sr, Er, 0), f32pair_to_f64(Si, Ei, 0));
        }
        if (VD) {
            // the channel's mu != 0 row: add its couplings to the mu = 0 functions
            float Sr = 0.f, Er = 0.f, Si = 0.f, Ei = 0.f;
#pragma unroll
            for (int s = 1; s < P; ++s) {
                const float4 v = vcs[ch * (P - 1) + s - 1];
                df_mac(v.x, v.y, zrh[s], zrl[s], Sr, Er);
                df_mac(-v.z, -v.w, zih[s], zil[s], Sr, Er);
                df_mac(v.x, v.y, zih[s], zil[s], Si, Ei);
                df_mac(v.z, v.w, zrh[s], zrl[s], Si, Ei);
            }
            double2 *y = Y + col * RSc + N0 + ch;
            const double2 y0 = *y;
            *y = make_double2(y0.x + f32pair_to_f64(Sr, Er, 0), y0.y + f32pair_to_f64(Si, Ei, 0));
        }
    }
}

// ------------------------------------------------------------- GEMM1
// Tile: 128 rows of A' (one q) x 128 columns of Z; K chunks of 32 (one
// 64-byte swizzled row per operand row), the four slices of both operands per
// stage, three stages; the four class accumulators fill TMEM (single buffer:
// the MMA warp waits for the epilogue to read a K group before the next).
// Each CTA loads the A and B tiles of its own output tile.
// K of each half: [kbeg, kbeg + klen); iq: the q of A.  half < 0: both K halves
// (complex v_t; row 2r of A' gives the real, 2r + 1 the imaginary part of row r
// of Y', so a warp's stores into one column of Y' are contiguous);
// half = 0 / 1 (real v_t): rows [0, D) of A' (U itself) against the real or
// imaginary half of the Z columns, giving the real or imaginary part of Y'.
struct G1Tile { int qslot, mrow, ncol0, klen, iq, kbeg, half; };

struct G1Params {
    const G1Tile *tiles;
    int ntiles;
    const QDesc *qd;
    const int *aexp;       // per A' row: [nk][MP]
    const int *zexp;       // per column of the batch
    double2 *Y;            // [col][RSc] (rows N0 + r)
    long long RSc;
    long long NC;          // columns of the batch (plane stride in rows of ZS)
    int RS, HS, MP, N0pad, Dpad, N0;
    int *err;
};

constexpr int G1_BM = 128, G1_BN = 128, G1_KC = 32;
constexpr int G1_A_PLANE = G1_BM * G1_KC * 2;              // 8 KB
constexpr int G1_B_PLANE = G1_BN * G1_KC * 2;              // 8 KB
constexpr int G1_STAGE = NPL * (G1_A_PLANE + G1_B_PLANE);   // 64 KB
constexpr int G1_STAGES = 3;
constexpr int G1_GROUP = 8;                                // chunks per exact K group (256)
constexpr int G1_TMEM = 512;                               // 4 classes x 128 columns
constexpr int G1_THREADS = 384;                            // 3 warpgroups
// register split (setmaxnreg): the control warpgroup gives its registers to
// the two epilogue warpgroups; 4*32*64 + 8*32*216 <= 12*32*168
constexpr int G1_REG_LAUNCH = 168, G1_REG_CTRL = 64, G1_REG_EPI = 216;
static_assert(4 * G1_REG_CTRL + 8 * G1_REG_EPI <= 12 * G1_REG_LAUNCH, "register split exceeds the launch allocation");

// warpgroup 0: warp 0 TMA producer, warp 1 MMA issuer (warps 2, 3 idle);
// warpgroups 1, 2: epilogue (TMEM lane quarter = w % 4, column half = (w - 4) / 4).
__global__ void __launch_bounds__(G1_THREADS, 1) gemm1_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB, G1Params p) {
    extern __shared__ __align__(1024) unsigned char g1_smem[];
    uintptr_t base = (reinterpret_cast<uintptr_t>(g1_smem) + 1023) & ~(uintptr_t)1023;
    unsigned char *stages = reinterpret_cast<unsigned char *>(base);
    __shared__ uint64_t full_bar[G1_STAGES], empty_bar[G1_STAGES], tfull_bar, tempty_bar, mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < G1_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&tfull_bar, 1);
        mbar_init(&tempty_bar, 8);
        mbar_init(&mma_done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_slot, G1_TMEM);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    uint32_t tmem = tmem_slot;

    if (warp < 4) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(G1_REG_CTRL));
        if (warp == 0 && lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            G1Tile nx = blockIdx.x < p.ntiles ? p.tiles[blockIdx.x] : G1Tile{};
            for (int t = blockIdx.x; t < p.ntiles && !abort_flag; t += gridDim.x) {
                const G1Tile tl = nx;
                // the next tile's descriptor, loaded now: its latency overlaps this tile's copies
                if (t + (int)gridDim.x < p.ntiles) nx = p.tiles[t + gridDim.x];
                const int qi = tl.iq;
                int nk = tl.klen / G1_KC;
                const int nchunk = tl.half < 0 ? 2 * nk : nk;
                bool stop = false;
                for (int kc = 0; kc < nchunk; ++kc) {
                    if (!mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, p.err, kDevTimeoutTma)) { stop = true; break; }
                    int xa = tl.kbeg + ((kc < nk) ? kc * G1_KC : p.HS + (kc - nk) * G1_KC), xb = xa;
                    if (tl.half >= 0) { xa = tl.kbeg + kc * G1_KC; xb = xa + tl.half * p.HS; }
                    unsigned char *st = stages + (size_t)s * G1_STAGE;
                    mbar_expect_tx(&full_bar[s], G1_STAGE);
#pragma unroll
                    for (int pl = 0; pl < NPL; ++pl) {
                        tma_load_2d(saddr(st + pl * G1_A_PLANE), &tmA, &full_bar[s], xa, (qi * NPL + pl) * p.MP + tl.mrow);
                        tma_load_2d(saddr(st + NPL * G1_A_PLANE + pl * G1_B_PLANE), &tmB, &full_bar[s], xb,
                                    (int)(pl * p.NC + tl.ncol0));
                    }
                    ++issued;
                    if (++s == G1_STAGES) { s = 0; ph ^= 1; }
                }
                if (stop) break;
            }
            if (abort_flag) {
                for (int i = 0; i < G1_STAGES && i < issued; ++i) mbar_drain(&full_bar[i], 0), mbar_drain(&full_bar[i], 1);
            }
        } else if (warp == 1 && lane == 0) {
            int s = 0;
            uint32_t ph = 0, eph = 0;
            // A slice a times B slices stacked in N (the B planes are contiguous)
            // lands in the class columns (a + b) G1_BN: six MMAs per K step cover
            // the ten slice products
            constexpr uint32_t id1 = idesc_bf16(G1_BM, G1_BN), id2 = idesc_bf16(G1_BM, 2 * G1_BN);
            bool ok = true;
            int nklen = blockIdx.x < p.ntiles ? p.tiles[blockIdx.x].klen : 0;
            int nhalf = blockIdx.x < p.ntiles ? p.tiles[blockIdx.x].half : -1;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
                const int klen = nklen, half = nhalf;
                if (t + (int)gridDim.x < p.ntiles) {   // prefetch
                    nklen = p.tiles[t + gridDim.x].klen;
                    nhalf = p.tiles[t + gridDim.x].half;
                }
                int nchunk = (half < 0 ? 2 : 1) * (klen / G1_KC);
                for (int g0 = 0; g0 < nchunk && ok; g0 += G1_GROUP) {
                    if (!mbar_wait(&tempty_bar, eph ^ 1, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                    tc_fence_after();
                    for (int kc = g0; kc < min(nchunk, g0 + G1_GROUP); ++kc) {
                        if (!mbar_wait(&full_bar[s], ph, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                        tc_fence_after();
                        unsigned char *st = stages + (size_t)s * G1_STAGE;
                        const uint32_t a0 = saddr(st), b0 = saddr(st + NPL * G1_A_PLANE);
                        const bool first = kc == g0;
#pragma unroll
                        for (int ks = 0; ks < G1_KC / 16; ++ks) {
                            const uint64_t d0 = desc_sw64(a0) + 2 * ks, d1 = desc_sw64(a0 + G1_A_PLANE) + 2 * ks;
                            const uint64_t d2 = desc_sw64(a0 + 2 * G1_A_PLANE) + 2 * ks;
                            const uint64_t d3 = desc_sw64(a0 + 3 * G1_A_PLANE) + 2 * ks;
                            const uint64_t e0 = desc_sw64(b0) + 2 * ks, e2 = desc_sw64(b0 + 2 * G1_B_PLANE) + 2 * ks;
                            const uint32_t acc = (first && ks == 0) ? 0u : 1u;   // the two a = 0 MMAs set all classes
                            umma_bf16(tmem, d0, e0, id2, acc);                    // classes 0, 1
                            umma_bf16(tmem + 2 * G1_BN, d0, e2, id2, acc);        // classes 2, 3
                            umma_bf16(tmem + G1_BN, d1, e0, id2, 1u);             // classes 1, 2
                            umma_bf16(tmem + 3 * G1_BN, d1, e2, id1, 1u);         // class 3
                            umma_bf16(tmem + 2 * G1_BN, d2, e0, id2, 1u);         // classes 2, 3
                            umma_bf16(tmem + 3 * G1_BN, d3, e0, id1, 1u);         // class 3
                        }
                        umma_commit(&empty_bar[s]);
                        if (++s == G1_STAGES) { s = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    umma_commit(&tfull_bar);
                    eph ^= 1;
                }
            }
            umma_drain(&mma_done);
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(G1_REG_EPI));
        const int quarter = warp % 4, half = (warp - 4) / 4;
        uint32_t eph = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            G1Tile tl = p.tiles[t];
            const QDesc q = p.qd[tl.qslot];
            int nchunk = (tl.half < 0 ? 2 : 1) * (tl.klen / G1_KC);
            int ngroups = (nchunk + G1_GROUP - 1) / G1_GROUP;
            // output scales: the row exponent, and the exponents of the 64 columns of
            // this half (lane l holds columns l and 32 + l; the store loop shuffles
            // them), fetched at tile start so that their latency overlaps the first
            // K group instead of following the last one
            const int r = tl.mrow + quarter * 32 + lane;     // row of A' in this q
            const bool im = tl.half < 0 ? (r & 1) : tl.half == 1;
            const int rr = tl.half < 0 ? (r >> 1) : r;
            const bool live = rr < q.D;
            const long long c0 = tl.ncol0 + half * 64, cend = q.colbase + q.ncols;
            const int ea = live ? p.aexp[(size_t)q.iq * p.MP + r] - 16 : 0;
            const int zx0 = c0 + lane < cend ? p.zexp[c0 + lane] : 0;
            const int zx1 = c0 + 32 + lane < cend ? p.zexp[c0 + 32 + lane] : 0;
            uint64_t hi[32], lo[32];   // packed pairs of columns
#pragma unroll
            for (int j = 0; j < 32; ++j) { hi[j] = 0; lo[j] = 0; }
            for (int gg = 0; gg < ngroups; ++gg) {
                if (!mbar_wait(&tfull_bar, eph, &abort_flag, p.err, kDevTimeoutEpi)) { ok = false; break; }
                tc_fence_after();
                uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + half * 64;
#pragma unroll
                for (int c0 = 0; c0 < 64; c0 += 8) {
                    uint32_t a0[8], a1[8], a2[8], a3[8];
                    tmem_ld8(tb + 0 * G1_BN + c0, a0);
                    tmem_ld8(tb + 1 * G1_BN + c0, a1);
                    tmem_ld8(tb + 2 * G1_BN + c0, a2);
                    tmem_ld8(tb + 3 * G1_BN + c0, a3);
                    tmem_wait_ld();
                    if (c0 + 8 == 64) {   // everything read: hand the accumulators back to the MMA warp
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty_bar);
                    }
#pragma unroll
                    for (int j = 0; j < 8; j += 2)
                        class_accumulate2(f2_pack(a0[j], a0[j + 1]), f2_pack(a1[j], a1[j + 1]), f2_pack(a2[j], a2[j + 1]),
                                          f2_pack(a3[j], a3[j + 1]), hi[(c0 + j) / 2], lo[(c0 + j) / 2]);
                }
                eph ^= 1;
            }
            if (!ok) break;
            double *dst = reinterpret_cast<double *>(p.Y + c0 * p.RSc + p.N0 + (live ? rr : 0)) + (im ? 1 : 0);
            const long long cstride = 2 * p.RSc;
#pragma unroll
            for (int j = 0; j < 64; j += 2) {
                const int e0 = __shfl_sync(0xffffffffu, j < 32 ? zx0 : zx1, j & 31);
                const int e1 = __shfl_sync(0xffffffffu, j + 1 < 32 ? zx0 : zx1, (j + 1) & 31);
                const float2 h = f2_unpack(hi[j / 2]), l = f2_unpack(lo[j / 2]);
                if (live && c0 + j < cend) dst[j * cstride] = f32pair_to_f64(h.x, l.x, ea + e0);
                if (live && c0 + j + 1 < cend) dst[(j + 1) * cstride] = f32pair_to_f64(h.y, l.y, ea + e1);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, G1_TMEM);
    }
}

// ------------------------------------------------------------- GEMM2
// bi2: the real form's second row block (-1: none); the complex form leaves it 0
struct G2Tile { int pair, bi, bj, bi2; };

struct G2Params {
    const G2Tile *tiles;
    int ntiles;
    const PairDesc *pairs;
    const QDesc *qd;
    const long long *praw_off;   // per pair, in doubles
    double *praw;
    const int *zexp, *yexp;      // per column of the batch
    long long NC;
    int HS, N0pad, nstages, stage_bytes;
    int fail_wait;               // test hook: the epilogue first waits on a barrier nothing completes
    int *err;
};

constexpr int G2_EPI_WARPS = 8;
constexpr int G2_MAX_STAGES = 4;

// K chunk of the Z^H Y tiles: 64 (128-byte swizzle) for band blocks up to 40,
// 32 (64-byte swizzle) above, so that at least three pipeline stages fit
__host__ __device__ constexpr int g2_kc(int NB) { return NB >= 48 ? 32 : 64; }

// number of K chunks of a pair: mu=0 rows plus the dense rows of its q
template <int KC> __device__ __forceinline__ int g2_chunks(const QDesc &q, int N0pad) { return (N0pad + q.D + KC - 1) / KC; }

// warp 0: TMA; warp 1: MMA; warps 2..9: epilogue (lane quarter = w%4,
// column half = (w-2)/4 of the W accumulator columns).  Four class
// accumulators of W columns each, single-buffered.
//
// Complex form (RE = false): A rows [0,NB) Re Z, [NB,2NB) Im Z of band block
// bi, B rows the same of Y block bj, K over each half: the W x W real
// embedding of P' (W = 2 NB).
// Real form (RE = true, inversion symmetry: two real bands per column, only
// Re P' = Zr^T Yr + Zi^T Yi is wanted): K runs over both halves of a column
// (2 x the chunks), A rows [0,NB) are Z block bi and [NB,2NB) block bi2, B rows
// Y block bj only (W = NB): half the MMA work.  Re P'[bi][bj] goes to the
// real-real quadrant of the complex tile layout.
template <int NB, bool RE>
__global__ void __launch_bounds__(64 + 32 * G2_EPI_WARPS, 1) gemm2_kernel(const __grid_constant__ CUtensorMap tmZ,
                                                                          const __grid_constant__ CUtensorMap tmY,
                                                                          G2Params p) {
    constexpr int KC = g2_kc(NB);                  // K values per chunk
    constexpr int G2_A_PLANE = 128 * KC * 2;       // rows [0, 2NB) loaded, rest zero
    constexpr int G2_GROUP = 256 / KC;             // chunks per exact K group (256)
    constexpr int W = RE ? NB : 2 * NB, CW = W / 2;   // accumulator columns; per thread
    constexpr int WT = 2 * NB;                     // output tile width of the complex layout
    constexpr int B_PLANE = W * KC * 2;
    static_assert(!RE || NB % 16 == 0, "the real form needs N = NB to be a multiple of 16");
    extern __shared__ __align__(1024) unsigned char g2_smem[];
    uintptr_t base = (reinterpret_cast<uintptr_t>(g2_smem) + 1023) & ~(uintptr_t)1023;
    unsigned char *stages = reinterpret_cast<unsigned char *>(base);
    __shared__ uint64_t full_bar[G2_MAX_STAGES], empty_bar[G2_MAX_STAGES], tfull_bar, tempty_bar, mma_done, never_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int NS = p.nstages, SB = p.stage_bytes;
    for (int s = 0; s < NS; ++s)
        for (int pl = 0; pl < NPL; ++pl) {
            uint4 *a = reinterpret_cast<uint4 *>(stages + (size_t)s * SB + pl * G2_A_PLANE);
            for (int i = threadIdx.x; i < G2_A_PLANE / 16; i += blockDim.x) a[i] = make_uint4(0, 0, 0, 0);
        }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&tfull_bar, 1);
        mbar_init(&tempty_bar, G2_EPI_WARPS);
        mbar_init(&mma_done, 1);
        mbar_init(&never_bar, 1);   // completed by nothing: the fault-injection wait
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) tmem_alloc(&tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    uint32_t tmem = tmem_slot;
    constexpr uint32_t box_bytes = (uint32_t)KC * NB * 2u;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            for (int t = blockIdx.x; t < p.ntiles && !abort_flag; t += gridDim.x) {
                G2Tile tl = p.tiles[t];
                const PairDesc pr = p.pairs[tl.pair];
                const QDesc q = p.qd[pr.qslot];
                int nc = g2_chunks<KC>(q, p.N0pad);
                const int nct = RE ? 2 * nc : nc;
                bool stop = false;
                for (int m = 0; m < pr.no && !stop; ++m) {
                    long long ya = pr.col0 + (long long)m * pr.nb + tl.bi * NB;
                    long long yb = pr.col0 + (long long)m * pr.nb + tl.bj * NB;
                    long long ya2 = pr.col0 + (long long)m * pr.nb + (tl.bi2 >= 0 ? tl.bi2 : tl.bi) * NB;
                    for (int c = 0; c < nct; ++c) {
                        if (!mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, p.err, kDevTimeoutTma)) { stop = true; break; }
                        unsigned char *st = stages + (size_t)s * SB;
                        mbar_expect_tx(&full_bar[s], (RE ? 3u : 4u) * NPL * box_bytes);
                        for (int pl = 0; pl < NPL; ++pl) {
                            unsigned char *a = st + pl * G2_A_PLANE;
                            unsigned char *b = st + NPL * G2_A_PLANE + pl * B_PLANE;
                            int ra = (int)(pl * p.NC + ya), rb = (int)(pl * p.NC + yb);
                            if constexpr (RE) {
                                // K over [Re half | Im half] of every column
                                const int x = c < nc ? c * KC : p.HS + (c - nc) * KC;
                                tma_load_2d(saddr(a), &tmZ, &full_bar[s], x, ra);
                                tma_load_2d(saddr(a + NB * KC * 2), &tmZ, &full_bar[s], x, (int)(pl * p.NC + ya2));
                                tma_load_2d(saddr(b), &tmY, &full_bar[s], x, rb);
                            } else {
                                tma_load_2d(saddr(a), &tmZ, &full_bar[s], c * KC, ra);
                                tma_load_2d(saddr(a + NB * KC * 2), &tmZ, &full_bar[s], p.HS + c * KC, ra);
                                tma_load_2d(saddr(b), &tmY, &full_bar[s], c * KC, rb);
                                tma_load_2d(saddr(b + NB * KC * 2), &tmY, &full_bar[s], p.HS + c * KC, rb);
                            }
                        }
                        ++issued;
                        if (++s == NS) { s = 0; ph ^= 1; }
                    }
                }
                if (stop) break;
            }
            if (abort_flag) {
                for (int i = 0; i < NS && i < issued; ++i) mbar_drain(&full_bar[i], 0), mbar_drain(&full_bar[i], 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t tph = 0;
            // A slice a times B slices stacked in N (the B planes are contiguous)
            // lands in the class columns (a + b) W: five (3 W <= 256) or six MMAs
            // per K step cover the ten slice products
            constexpr uint32_t id1 = idesc_bf16(128, W), id2 = idesc_bf16(128, 2 * W);
            constexpr bool three = 3 * W <= 256;
            constexpr uint32_t id3 = idesc_bf16(128, three ? 3 * W : W);
            bool ok = true;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
                G2Tile tl = p.tiles[t];
                const PairDesc pr = p.pairs[tl.pair];
                const QDesc q = p.qd[pr.qslot];
                int nc = (RE ? 2 : 1) * g2_chunks<KC>(q, p.N0pad);
                for (int m = 0; m < pr.no && ok; ++m) {
                    for (int g0 = 0; g0 < nc && ok; g0 += G2_GROUP) {
                        if (!mbar_wait(&tempty_bar, tph ^ 1, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                        tc_fence_after();
                        for (int c = g0; c < min(nc, g0 + G2_GROUP); ++c) {
                            if (!mbar_wait(&full_bar[s], ph, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                            tc_fence_after();
                            unsigned char *st = stages + (size_t)s * SB;
                            uint32_t a0 = saddr(st), b0 = saddr(st + NPL * G2_A_PLANE);
#pragma unroll
                            for (int ks = 0; ks < KC / 16; ++ks) {
                                // K-major operands, 128- or 64-byte swizzle (one swizzled row per chunk)
                                auto dsc = [](uint32_t a) { return KC == 64 ? desc_sw128(a) : desc_sw64(a); };
                                const uint64_t d0 = dsc(a0) + 2 * ks, d1 = dsc(a0 + G2_A_PLANE) + 2 * ks;
                                const uint64_t d2 = dsc(a0 + 2 * G2_A_PLANE) + 2 * ks;
                                const uint64_t d3 = dsc(a0 + 3 * G2_A_PLANE) + 2 * ks;
                                const uint64_t e0 = dsc(b0) + 2 * ks, e2 = dsc(b0 + 2 * B_PLANE) + 2 * ks;
                                const uint32_t acc = (c == g0 && ks == 0) ? 0u : 1u;   // the two a = 0 MMAs set all classes
                                umma_bf16(tmem, d0, e0, id2, acc);                  // classes 0, 1
                                umma_bf16(tmem + 2 * W, d0, e2, id2, acc);          // classes 2, 3
                                if (three) {
                                    umma_bf16(tmem + W, d1, e0, id3, 1u);           // classes 1, 2, 3
                                } else {
                                    umma_bf16(tmem + W, d1, e0, id2, 1u);           // classes 1, 2
                                    umma_bf16(tmem + 3 * W, d1, e2, id1, 1u);       // class 3
                                }
                                umma_bf16(tmem + 2 * W, d2, e0, id2, 1u);           // classes 2, 3
                                umma_bf16(tmem + 3 * W, d3, e0, id1, 1u);           // class 3
                            }
                            umma_commit(&empty_bar[s]);
                            if (++s == NS) { s = 0; ph ^= 1; }
                        }
                        if (!ok) break;
                        umma_commit(&tfull_bar);
                        tph ^= 1;
                    }
                }
            }
            umma_drain(&mma_done);
        }
    } else {
        int e = warp - 2;
        int quarter = warp % 4, cg = e / 4;
        uint32_t tph = 0;
        bool ok = true;
        // accumulator row: complex form Re (< NB) or Im part of band bi*NB + row % NB;
        // real form band bi*NB + row (< NB) or bi2*NB + row - NB
        int row = quarter * 32 + lane;
        // fault-injection hook: a bounded wait of about 1 ms that nothing completes
        if (p.fail_wait && !mbar_wait_ns(&never_bar, 0, &abort_flag, p.err, kDevTimeoutEpi, 1000000ULL)) ok = false;
        for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            G2Tile tl = p.tiles[t];
            const PairDesc pr = p.pairs[tl.pair];
            const QDesc q = p.qd[pr.qslot];
            int nc = (RE ? 2 : 1) * g2_chunks<KC>(q, p.N0pad);
            const int brow = (RE && row >= NB) ? (tl.bi2 >= 0 ? tl.bi2 : tl.bi) : tl.bi;
            uint64_t hi[CW / 2], lo[CW / 2];   // packed pairs of columns
#pragma unroll
            for (int j = 0; j < CW / 2; ++j) { hi[j] = 0; lo[j] = 0; }
            for (int m = 0; m < pr.no && ok; ++m) {
                long long cola = pr.col0 + (long long)m * pr.nb + brow * NB + (row % NB);
                long long colb0 = pr.col0 + (long long)m * pr.nb + tl.bj * NB;
                int ea = p.zexp[min(cola, p.NC - 1)] - 16;
                // exponents of the NB columns of Y, fetched once per m: lane l holds
                // columns l and 32 + l (the drain loop shuffles them)
                const int yx0 = p.yexp[min(colb0 + lane, p.NC - 1)];
                const int yx1 = p.yexp[min(colb0 + 32 + lane, p.NC - 1)];
                for (int g0 = 0; g0 < nc; g0 += G2_GROUP) {
                    if (!mbar_wait(&tfull_bar, tph, &abort_flag, p.err, kDevTimeoutEpi)) { ok = false; break; }
                    tc_fence_after();
                    uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + cg * CW;
#pragma unroll
                    for (int c0 = 0; c0 < CW; c0 += 8) {
                        uint32_t a0[8], a1[8], a2[8], a3[8];
                        tmem_ld8(tb + 0 * W + c0, a0);
                        tmem_ld8(tb + 1 * W + c0, a1);
                        tmem_ld8(tb + 2 * W + c0, a2);
                        tmem_ld8(tb + 3 * W + c0, a3);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 8; j += 2) {
                            const int b = cg * CW + c0 + j, j0 = b % NB, j1 = (b + 1) % NB;
                            const float s0 = ldexpf(1.0f, ea + __shfl_sync(0xffffffffu, j0 < 32 ? yx0 : yx1, j0 & 31));
                            const float s1 = ldexpf(1.0f, ea + __shfl_sync(0xffffffffu, j1 < 32 ? yx0 : yx1, j1 & 31));
                            class_accumulate2_sc(f2_pack(a0[j], a0[j + 1]), f2_pack(a1[j], a1[j + 1]),
                                                 f2_pack(a2[j], a2[j + 1]), f2_pack(a3[j], a3[j + 1]),
                                                 f2_pack(__float_as_uint(s0), __float_as_uint(s1)), hi[(c0 + j) / 2],
                                                 lo[(c0 + j) / 2]);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty_bar);
                    tph ^= 1;
                }
            }
            if (!ok) break;
            const bool store = RE ? (row < NB || (row < 2 * NB && tl.bi2 >= 0)) : row < W;
            if (store) {
                int nblk = (pr.nb + NB - 1) / NB;
                double *out = p.praw + p.praw_off[tl.pair] + ((size_t)brow * nblk + tl.bj) * WT * WT +
                              (size_t)(RE ? row % NB : row) * WT + cg * CW;
#pragma unroll
                for (int j = 0; j < CW; j += 2) {
                    const float2 h = f2_unpack(hi[j / 2]), l = f2_unpack(lo[j / 2]);
                    out[j] = f32pair_to_f64(h.x, l.x, 0);
                    out[j + 1] = f32pair_to_f64(h.y, l.y, 0);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

}  // namespace

namespace tc {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult qr;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}

// 2-D BF16 tensor [rows][cols] (cols contiguous), box {64, box_rows}, 128-byte swizzle
int make_map_2d(hfx_ctx *ctx, CUtensorMap *m, const void *ptr, long long rows, long long cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_err(ctx, HFX_EDEVICE, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_err(ctx, HFX_EDEVICE, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return HFX_OK;
}

// 2-D BF16 tensor [rows][cols], box {box_cols, box_rows}, swizzle of box_cols*2 bytes (32, 64 or 128)
int make_map_2d_sw(hfx_ctx *ctx, CUtensorMap *m, const void *ptr, long long rows, long long cols, int box_rows,
                   int box_cols, int swizzle_bytes) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_err(ctx, HFX_EDEVICE, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUtensorMapSwizzle sw = swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                            : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                            : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE;
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_err(ctx, HFX_EDEVICE, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return HFX_OK;
}

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace tc

template <typename V>
void launch_slice_cols(const V *d_Z, long long RSc, const QDesc *d_q, int nq, long long NC, long long maxcols, int N0,
                       int N0pad, int Dpad, int RS, __nv_bfloat16 *d_XS, int *d_exp, cudaStream_t st) {
    long long g = (maxcols + 7) / 8;
    if (g > 8192) g = 8192;
    if (g < 1) g = 1;
    dim3 grid((unsigned)g, (unsigned)nq);
    slice_cols_kernel<V><<<grid, 256, 0, st>>>(d_Z, RSc, d_q, N0, N0pad, Dpad, RS, NC, d_XS, d_exp);
}
template void launch_slice_cols<float2>(const float2 *, long long, const QDesc *, int, long long, long long, int, int,
                                        int, int, __nv_bfloat16 *, int *, cudaStream_t);
template void launch_slice_cols<double2>(const double2 *, long long, const QDesc *, int, long long, long long, int, int,
                                         int, int, __nv_bfloat16 *, int *, cudaStream_t);

bool block_y_couples(int P, int N0) { return P >= 2 && P <= 4 && N0 > 0 && N0 % (P - 1) == 0; }

template <typename V>
void launch_block_y(const QDesc *d_q, int nq, const double2 *const *d_VB, const double2 *const *d_VD, const V *d_Z,
                    double2 *d_Y, long long RSc, int P, int N0, long long maxcols, cudaStream_t st) {
    if (N0 == 0 || nq == 0) return;
    long long per = maxcols * N0;
    long long g = (per + 255) / 256;
    if (g > 8192) g = 8192;
    dim3 grid((unsigned)g, (unsigned)nq);
    if constexpr (std::is_same<V, double2>::value) {
        if (block_y_couples(P, N0)) {
            const long long per_df = maxcols * (N0 / (P - 1));
            const dim3 grid_df((unsigned)std::min<long long>(8192, (per_df + 255) / 256), (unsigned)nq);
            const size_t sm = (size_t)N0 * (P + 1) * sizeof(float4);
            if (P == 2) block_y_df_kernel<2><<<grid_df, 256, sm, st>>>(d_q, d_VB, d_VD, d_Z, d_Y, RSc, N0);
            else if (P == 3) block_y_df_kernel<3><<<grid_df, 256, sm, st>>>(d_q, d_VB, d_VD, d_Z, d_Y, RSc, N0);
            else block_y_df_kernel<4><<<grid_df, 256, sm, st>>>(d_q, d_VB, d_VD, d_Z, d_Y, RSc, N0);
            return;
        }
    }
    block_y_kernel<V><<<grid, 256, 0, st>>>(d_q, d_VB, d_Z, d_Y, RSc, P, N0);
}
template void launch_block_y<float2>(const QDesc *, int, const double2 *const *, const double2 *const *, const float2 *,
                                     double2 *, long long, int, int, long long, cudaStream_t);
template void launch_block_y<double2>(const QDesc *, int, const double2 *const *, const double2 *const *,
                                      const double2 *, double2 *, long long, int, int, long long, cudaStream_t);

// Tiles of GEMM1 for one batch.  The A operand is the upper triangle U of the
// dense block, so a row tile's K range (in each half) starts at its first row:
// [N0pad + r_min, N0pad + D), rounded to the K chunk.  Order, per q: groups of
// G1_COLGROUP 128-column blocks; inside a group, every row tile for each block
// of the group in turn.  The tiles running at once then share a few A row tiles
// and a few Z column blocks, both of which stay in L2 (the A slices of one q
// are up to ~140 MB on the largest workloads, more than L2), and the Re and Im
// rows of one Y column meet in L2.
constexpr int G1_COLGROUP = 8;
int gemm1_tiles(const QDesc *h_q, int nq, int N0pad, bool real_v, std::vector<unsigned char> &out) {
    std::vector<G1Tile> tiles;
    for (int s = 0; s < nq; ++s) {
        const QDesc &q = h_q[s];
        // row tiles over the 2 D interleaved real and imaginary rows; with a real
        // v_t over the D rows of U, each taken once per half of the Z columns
        const int rows = real_v ? q.D : 2 * q.D;
        const int mt = (rows + G1_BM - 1) / G1_BM;
        std::vector<int> kbeg(mt), klen(mt);
        for (int i = 0; i < mt; ++i) {
            const int r0 = i * G1_BM;   // rows [r0, r0 + 128) of A': rows r0 / 2 .. of U when interleaved
            const int rmin = real_v ? r0 : r0 / 2;
            kbeg[i] = N0pad + rmin / G1_KC * G1_KC;
            klen[i] = (N0pad + q.D - kbeg[i] + G1_KC - 1) / G1_KC * G1_KC;
        }
        for (long long g0 = 0; g0 < q.ncols; g0 += (long long)G1_BN * G1_COLGROUP)
            for (int i = 0; i < mt; ++i)
                for (int h = real_v ? 0 : -1; h < (real_v ? 2 : 0); ++h)
                    for (int j = 0; j < G1_COLGROUP; ++j) {
                        const long long n0 = g0 + (long long)j * G1_BN;
                        if (n0 < q.ncols)
                            tiles.push_back(G1Tile{s, i * G1_BM, (int)(q.colbase + n0), klen[i], q.iq, kbeg[i], h});
                    }
    }
    out.assign(reinterpret_cast<const unsigned char *>(tiles.data()),
               reinterpret_cast<const unsigned char *>(tiles.data()) + tiles.size() * sizeof(G1Tile));
    return (int)tiles.size();
}

int launch_gemm1_tc(hfx_ctx *ctx, const __nv_bfloat16 *d_Ap_all, long long ap_rows, const int *d_aexp, const QDesc *d_q,
                    const __nv_bfloat16 *d_ZS, const int *d_zexp, double2 *d_Y, long long RSc, long long NC, int N0,
                    int N0pad, int Dpad, int RS, const void *d_tiles, int ntiles) {
    int HS = N0pad + Dpad, MP = 2 * Dpad;
    if (ntiles == 0) return HFX_OK;
    if (NC > 0x7fffffffLL / 4) return set_err(ctx, HFX_EUNSUPPORTED, "batch has too many columns for 32-bit TMA coordinates");
    int rc;
    CUtensorMap mA, mB;
    if ((rc = make_map_2d_sw(ctx, &mA, d_Ap_all, ap_rows, RS, G1_BM, G1_KC, 64))) return rc;
    if ((rc = make_map_2d_sw(ctx, &mB, d_ZS, (long long)NPL * NC, RS, G1_BN, G1_KC, 64))) return rc;
    G1Params p;
    p.tiles = reinterpret_cast<const G1Tile *>(d_tiles);
    p.ntiles = ntiles;
    p.qd = d_q;
    p.aexp = d_aexp;
    p.zexp = d_zexp;
    p.Y = d_Y;
    p.RSc = RSc;
    p.N0 = N0;
    p.NC = NC;
    p.RS = RS;
    p.HS = HS;
    p.MP = MP;
    p.N0pad = N0pad;
    p.Dpad = Dpad;
    p.err = ctx->d_err;
    size_t smem = (size_t)G1_STAGES * G1_STAGE + 1024;
    auto kern = gemm1_kernel;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    {
        // the register split of the kernel assumes this launch allocation
        cudaFuncAttributes fa;
        if ((rc = cuda_check(ctx, cudaFuncGetAttributes(&fa, kern), "gemm1 attributes"))) return rc;
        if (fa.numRegs < G1_REG_LAUNCH)
            return set_err(ctx, HFX_EUNSUPPORTED, "gemm1 compiled with fewer registers than its warpgroup split needs");
    }
    const int grid = std::min<int>(num_sms(), ntiles);
    kern<<<grid, G1_THREADS, smem, ctx->stream>>>(mA, mB, p);
    return cuda_check(ctx, cudaGetLastError(), "gemm1 launch");
}

// Tiles of GEMM2: every (band block i, band block j) of every pair with
// occupied bands at k - q.
int gemm2_tiles(const PairDesc *h_pairs, int npairs, int NB, bool real_form, std::vector<unsigned char> &out) {
    std::vector<G2Tile> tiles;
    for (int i = 0; i < npairs; ++i) {
        int nblk = (h_pairs[i].nb + NB - 1) / NB;
        if (h_pairs[i].no == 0) continue;
        if (real_form) {   // two row blocks per tile
            for (int bi = 0; bi < nblk; bi += 2)
                for (int bj = 0; bj < nblk; ++bj) tiles.push_back(G2Tile{i, bi, bj, bi + 1 < nblk ? bi + 1 : -1});
        } else {
            for (int bi = 0; bi < nblk; ++bi)
                for (int bj = 0; bj < nblk; ++bj) tiles.push_back(G2Tile{i, bi, bj, 0});
        }
    }
    out.assign(reinterpret_cast<const unsigned char *>(tiles.data()),
               reinterpret_cast<const unsigned char *>(tiles.data()) + tiles.size() * sizeof(G2Tile));
    return (int)tiles.size();
}

int gemm2_check_nb(int NB) { return NB % 8 == 0 && NB >= 8 && NB <= 64; }
bool gemm2_real_form(int NB) { return NB % 16 == 0; }

int launch_gemm2_tc(hfx_ctx *ctx, const __nv_bfloat16 *d_ZS, const __nv_bfloat16 *d_YS, const int *d_zexp,
                    const int *d_yexp, long long NC, int RS, int HS, int N0pad, const PairDesc *d_pairs, const QDesc *d_q,
                    int NB, const long long *d_praw_off, double *d_praw, const void *d_tiles, int ntiles, int fail_wait,
                    bool real_form) {
    if (real_form && !gemm2_real_form(NB)) return set_err(ctx, HFX_EINVAL, "gemm2: the real form needs a band tile of 16, 32, 48 or 64");
    if (!gemm2_check_nb(NB)) return set_err(ctx, HFX_EINVAL, "gemm2: band tile must be a multiple of 8 up to 64");
    if (ntiles == 0) return HFX_OK;
    if (NC > 0x7fffffffLL / 4) return set_err(ctx, HFX_EUNSUPPORTED, "batch has too many columns for 32-bit TMA coordinates");
    int rc;
    CUtensorMap mZ, mY;
    const int KC = g2_kc(NB);
    if ((rc = make_map_2d_sw(ctx, &mZ, d_ZS, (long long)NPL * NC, RS, NB, KC, 2 * KC))) return rc;
    if ((rc = make_map_2d_sw(ctx, &mY, d_YS, (long long)NPL * NC, RS, NB, KC, 2 * KC))) return rc;
    G2Params p;
    p.tiles = reinterpret_cast<const G2Tile *>(d_tiles);
    p.ntiles = ntiles;
    p.pairs = d_pairs;
    p.qd = d_q;
    p.praw_off = d_praw_off;
    p.praw = d_praw;
    p.zexp = d_zexp;
    p.yexp = d_yexp;
    p.NC = NC;
    p.HS = HS;
    p.N0pad = N0pad;
    p.fail_wait = fail_wait;
    p.err = ctx->d_err;
    p.stage_bytes = NPL * (128 * KC * 2 + (real_form ? 1 : 2) * NB * KC * 2);
    p.nstages = std::min(G2_MAX_STAGES, (int)((226 * 1024) / p.stage_bytes));
    if (p.nstages < 1) return set_err(ctx, HFX_EUNSUPPORTED, "gemm2 stage does not fit in shared memory");
    size_t smem = (size_t)p.nstages * p.stage_bytes + 1024;
    int grid = std::min<int>(num_sms(), p.ntiles);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, 64 + 32 * G2_EPI_WARPS, smem, ctx->stream>>>(mZ, mY, p);
    };
    if (real_form) {
        switch (NB) {
        case 16: go(gemm2_kernel<16, true>); break;
        case 32: go(gemm2_kernel<32, true>); break;
        case 48: go(gemm2_kernel<48, true>); break;
        default: go(gemm2_kernel<64, true>); break;
        }
    } else {
        switch (NB) {
        case 8: go(gemm2_kernel<8, false>); break;
        case 16: go(gemm2_kernel<16, false>); break;
        case 24: go(gemm2_kernel<24, false>); break;
        case 32: go(gemm2_kernel<32, false>); break;
        case 40: go(gemm2_kernel<40, false>); break;
        case 48: go(gemm2_kernel<48, false>); break;
        case 56: go(gemm2_kernel<56, false>); break;
        default: go(gemm2_kernel<64, false>); break;
        }
    }
    return cuda_check(ctx, cudaGetLastError(), "gemm2 launch");
}

}  // namespace hfx
