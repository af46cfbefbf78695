// k_zipw_tc.cu -- interstitial projections on the tensor cores.
//
//   Z_kq[G, m, n] = Omega^{-1/2} sum_{G1 in k'} conj(c_{G1}(m, k')) T_n(G + G1 - G0)   (Sec. III.B)
//
// For a fixed k and a fixed shift W = G - G0, every (k', m) row of every pair
// (k, q) that needs this W is one row of a GEMM
//   Z[(k', m), n] = sum_{G1} C[(k', m), G1] T_k[n](W + G1),   C = conj(c),
// whose reduction index G1 runs over the plane waves of all k' in segments of
// 4 consecutive z values along the (x, y) lines of the plane-wave spheres.
//
// Operands (fixed-point slices of tc_ptx.cuh, real embedding of the complex
// product with the real and imaginary outputs side by side in N); one segment
// is 8 K values, the real and imaginary parts of its 4 z values:
//   A row (k', m) = [ Re C(4 z) | Im C(4 z) ] per segment   (128-byte swizzle, 2-D TMA)
//   B rows        = [ T_r(4 z) | -T_i(4 z) ] (real out), [ T_i(4 z) | T_r(4 z) ] (imag out)
// The sliced T box is stored in blocks of 4 z with all planes and both output
// rows of all bands of a band block contiguous, so the B operand of one
// segment is a single 1-D bulk copy (no swizzle).  A copy must start on a
// 16-byte boundary, i.e. at a multiple of 4 in z: T is kept in four copies
// shifted by 0, 1, 2, 3 in z, so a segment may start at any z.
#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "tc_ptx.cuh"

namespace hfx {

using namespace tc;

namespace {

constexpr int ZT_BM = 128;
// K chunk: KSEG segments of 8 K values.  Band blocks up to 40 take 8 segments
// (64 K, 128-byte swizzle, two stages); larger ones 4 (32 K, 64-byte swizzle,
// three stages), so that the stages of a 64-band tile still fit
__host__ __device__ constexpr int zt_kseg(int NB) { return NB > 40 ? 4 : 8; }
__host__ __device__ constexpr int zt_stages(int KSEG) { return KSEG == 8 ? 2 : 3; }
constexpr int ZT_EPI = 8;
constexpr int ZT_THREADS = 128 + 32 * ZT_EPI;   // warpgroup 0: producer, MMA (2 idle); 1, 2: epilogue
// register split (setmaxnreg) for the band blocks whose epilogue needs more than
// the 168 registers a thread gets at launch: the control warpgroup gives its
// registers to the two epilogue warpgroups (4*32*64 + 8*32*216 <= 12*32*168)
__host__ __device__ constexpr bool zt_split(int NB) { return NB >= 56; }
constexpr int ZT_REG_LAUNCH = 168, ZT_REG_CTRL = 64, ZT_REG_EPI = 216;
static_assert(4 * ZT_REG_CTRL + 8 * ZT_REG_EPI <= 12 * ZT_REG_LAUNCH, "register split exceeds the launch allocation");
constexpr int ZT_SEGZ = 4;                 // z values per segment (8 K values: real and imaginary parts)
constexpr int ZT_NCOPY = ZT_SEGZ;          // z-shifted copies of the sliced T box

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ------------------------------------------------------------- C slices
// One block per row r = (k', m) of c scaled by Omega^{-1/2}: exponent over
// |Re c|, |Im c| of the row, then
// Re C = c_r at K = 8 s + j and Im C = -c_i at K = 8 s + 4 + j, where segment
// s = segstart + (z - z0) / 4 and j = (z - z0) mod 4 on the segment grid of the
// row's tile.
__global__ void c_slices_kernel(const double2 *const *__restrict__ ck, const int *const *__restrict__ Gk,
                                const int *__restrict__ npw_k, const int *__restrict__ rowk, const int *__restrict__ rowm,
                                const int *__restrict__ line_of, int gx0, int gy0, int By, int nL,
                                const int *__restrict__ segstart, const int *__restrict__ segz0, int Kp, int Rpad,
                                double rs, __nv_bfloat16 *__restrict__ A, int *__restrict__ aexp) {
    int r = blockIdx.x;
    int kp = rowk[r], m = rowm[r];
    int npw = npw_k[kp];
    const double2 *c = ck[kp] + (size_t)m * npw;
    const int *G = Gk[kp];
    __shared__ unsigned long long red[256];
    unsigned long long mx = 0;
    for (int i = threadIdx.x; i < npw; i += blockDim.x) mx = max(mx, max(abs_bits(rs * c[i].x), abs_bits(rs * c[i].y)));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    int e = line_exp_bits(red[0]);
    if (threadIdx.x == 0) aexp[r] = e;
    // the whole A buffer is zeroed before this kernel: only the plane waves are written
    for (int i = threadIdx.x; i < npw; i += blockDim.x) {
        int li = line_of[(G[3 * i] - gx0) * By + (G[3 * i + 1] - gy0)];
        int z = G[3 * i + 2];
        __nv_bfloat16 sr[NPL], si[NPL];
        slice4(rs * c[i].x, e, sr);
        slice4(-(rs * c[i].y), e, si);
        const size_t sl = (size_t)(r / ZT_BM) * nL + li;   // segment grid of the row's tile
        const int dz = z - segz0[sl];
        const long long K = (long long)(segstart[sl] + dz / ZT_SEGZ) * 8 + dz % ZT_SEGZ;
#pragma unroll
        for (int p = 0; p < NPL; ++p) {
            __nv_bfloat16 *row = A + ((long long)p * Rpad + r) * Kp;
            row[K] = sr[p];
            row[K + ZT_SEGZ] = si[p];
        }
    }
}

// ------------------------------------------------------------- T slices
// Band exponents: grid (n, k) over the bands, max over the box of T_k[n].
__global__ void t_exp_kernel(const double2 *const *__restrict__ Tk, const int *__restrict__ nb_k, int td0, int td1,
                             int td2, int nbmax, const int *__restrict__ kslot, int *__restrict__ eT) {
    int n = blockIdx.x, k = blockIdx.y;
    if (kslot[k] < 0 || n >= nb_k[k]) return;
    long long box = (long long)td0 * td1 * td2;
    const double2 *T = Tk[k] + (size_t)n * box;
    __shared__ unsigned long long red[256];
    unsigned long long mx = 0;
    for (long long i = threadIdx.x; i < box; i += blockDim.x) mx = max(mx, max(abs_bits(T[i].x), abs_bits(T[i].y)));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) eT[(size_t)k * nbmax + n] = line_exp_bits(red[0]);
}

// Slices of T: one thread per (k, cell (X, Y, zb), band n) slices the 7 values
// T_k[n](X, Y, 4 zb .. 4 zb + 6) once and writes, for every copy c (T shifted
// by c in z) and plane p, the two B rows of band n = b NB + j over the 4 z
// values 4 zb + c .. 4 zb + c + 3:
//   Tq[c][k][X][Y][zb][b][p][j]      = [ Re T (4 z) | -Im T (4 z) ]   (real output)
//   Tq[c][k][X][Y][zb][b][p][NB + j] = [ Im T (4 z) |  Re T (4 z) ]   (imaginary output)
// (16 bytes each); bands past nb(k) and z past the box are 0.  Consecutive
// threads take consecutive bands, so the row stores are coalesced.  One
// (c, k, X, Y, zb, b) block -- all planes of one segment -- is contiguous.
__global__ void t_slices_kernel(const double2 *const *__restrict__ Tk, const int *__restrict__ nb_k, int td0, int td1,
                                int td2, int nzb, int NB, int nblk, int nbmax, int nslot, const int *__restrict__ kslot,
                                const int *__restrict__ eT, __nv_bfloat16 *__restrict__ Tq) {
    constexpr int NZ = ZT_SEGZ + ZT_NCOPY - 1;                // z values a thread needs
    const int k = blockIdx.y;
    const int slot = kslot[k];
    if (slot < 0) return;
    const int nbpad = NB * nblk;
    const long long ncell = (long long)td0 * td1 * nzb;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ncell * nbpad) return;
    const int n = (int)(idx % nbpad);
    const long long cellk = idx / nbpad;                      // (X, Y, zb) of this k
    const int zb = (int)(cellk % nzb);
    const long long xy = cellk / nzb;
    const bool live = n < nb_k[k];
    const long long box = (long long)td0 * td1 * td2;
    const double2 *T = live ? Tk[k] + (size_t)n * box + xy * td2 : nullptr;
    const int e = live ? eT[(size_t)k * nbmax + n] : 0;
    __nv_bfloat16 sr[NZ][NPL], si[NZ][NPL];
#pragma unroll
    for (int t = 0; t < NZ; ++t) {
        const int z = zb * ZT_SEGZ + t;
        const double2 v = (live && z < td2) ? T[z] : make_double2(0.0, 0.0);
        slice4(v.x, e, sr[t]);
        slice4(v.y, e, si[t]);
    }
    const int b = n / NB, j = n % NB;
    const long long blk = 2LL * NB * 8;                       // one plane of a block: 2 NB rows of 8 values
#pragma unroll
    for (int c = 0; c < ZT_NCOPY; ++c) {
        const long long cell = ((long long)c * nslot + slot) * ncell + cellk;
        __nv_bfloat16 *dst = Tq + (cell * nblk + b) * (NPL * blk) + (long long)j * 8;
#pragma unroll
        for (int p = 0; p < NPL; ++p) {
            uint4 ro, io;   // real-output row, imaginary-output row
            ro.x = pack_bf16x2(sr[c][p], sr[c + 1][p]);
            ro.y = pack_bf16x2(sr[c + 2][p], sr[c + 3][p]);
            ro.z = pack_bf16x2(__hneg(si[c][p]), __hneg(si[c + 1][p]));
            ro.w = pack_bf16x2(__hneg(si[c + 2][p]), __hneg(si[c + 3][p]));
            io.x = pack_bf16x2(si[c][p], si[c + 1][p]);
            io.y = pack_bf16x2(si[c + 2][p], si[c + 3][p]);
            io.z = ro.x;
            io.w = ro.y;
            *reinterpret_cast<uint4 *>(dst + p * blk) = ro;
            *reinterpret_cast<uint4 *>(dst + p * blk + NB * 8) = io;
        }
    }
}

// ------------------------------------------------------------- GEMM
struct ZTile { int k, w, mrow, nblk; };

struct ZPairInfo { int pair; int g0x, g0y, g0z; };

struct ZParams {
    const ZTile *tiles;
    int ntiles;
    const int4 *wxyz;             // [nw] shift W (x, y, z)
    const ZPairInfo *pinfo;       // [nk][nk] by (k, k')
    const PairDesc *pairs;
    const int *gtab;              // [nq][ax][ay][az] aux index or -1
    int ax0, ay0, az0, ad0, ad1, ad2;
    const int *rowk, *rowm;       // rows of A (k', m)
    const int *aexp, *eT;         // row exponents, [k][n] band exponents
    const int *kslot;             // k -> slot of its T slices
    const int2 *segoff;           // [row tile][segment] (x td1 + y of its line, z0)
    int nsegp_max;
    const int *nchunk;            // [row tile] 64-K chunks
    const int *runs;              // [row tile][chunk] bit j: segment j of the chunk starts a bulk copy; bits 8..: live segments
    const __nv_bfloat16 *Tq;      // sliced T blocks (t_slices_kernel layout)
    int td0, td1, nzb, nblk, nslot;
    double2 *ZI;                  // output plane ZI[g][col] (rows g of the interstitial part, G-major)
    long long NCi;                // row stride of ZI: the columns of the batch
    int nmt, nk, R, Rpad, nbmax, tlo0, tlo1, tlo2;
    double rs;                    // Omega^{-1/2}
    int *err;
};

// warp 0: TMA; warp 1: MMA; warps 4..11: epilogue (lane quarter, real/imaginary output)
template <int NB>
__global__ void __launch_bounds__(ZT_THREADS, 1) zipw_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                      ZParams p) {
    constexpr int N = 2 * NB;                            // real and imaginary output columns
    constexpr int KSEG = zt_kseg(NB);                    // segments per K chunk
    constexpr int KC = 8 * KSEG;                         // K values per chunk
    constexpr int ZT_A_PLANE = 128 * KC * 2;             // 128 rows x KC K
    constexpr int ZT_GROUP = 256 / KC;                   // chunks per exact group (256)
    constexpr int ZT_STAGES = zt_stages(KSEG);
    constexpr int SEGB = N * 16;                         // one segment of one plane: N rows x 8 K
    constexpr int SEG4 = NPL * SEGB;                     // one segment, all planes (one bulk copy)
    constexpr int STAGE = NPL * ZT_A_PLANE + KSEG * SEG4;   // KSEG segments per chunk
    extern __shared__ __align__(1024) unsigned char zt_smem[];
    uintptr_t base = (reinterpret_cast<uintptr_t>(zt_smem) + 1023) & ~(uintptr_t)1023;
    unsigned char *stages = reinterpret_cast<unsigned char *>(base);
    __shared__ uint64_t full_bar[ZT_STAGES], empty_bar[ZT_STAGES], tfull_bar, tempty_bar, mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    __shared__ int s_eT[ZT_EPI][32];      // per epilogue warp: the band exponents of its bands
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // B segments of every stage start as zeros: padding segments are never loaded
    for (int s = 0; s < ZT_STAGES; ++s) {
        uint4 *bz = reinterpret_cast<uint4 *>(stages + (size_t)s * STAGE + NPL * ZT_A_PLANE);
        for (int i = threadIdx.x; i < KSEG * SEG4 / 16; i += blockDim.x) bz[i] = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int s = 0; s < ZT_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&tfull_bar, 1);
        mbar_init(&tempty_bar, ZT_EPI);
        mbar_init(&mma_done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    uint32_t tmem = tmem_slot;

    if (warp < 4) {
    if constexpr (zt_split(NB)) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(ZT_REG_CTRL));
    if (warp == 0) {
        // producer warp: lane 0 waits for the stage and arms its barrier, then
        // lanes 0..3 load the four A planes and the lanes of the segments that
        // start a run (consecutive z blocks of one line, contiguous in T) one
        // bulk copy each; padding segments are not loaded (their A is zero and
        // their shared memory holds finite data of earlier chunks or zeros)
        int s = 0;
        uint32_t ph = 0;
        int issued = 0;
        const char *tq = reinterpret_cast<const char *>(p.Tq);
        // the tables of the next chunk (and the next tile's descriptor) are loaded
        // one step ahead, so that their latency overlaps the wait for a free stage
        ZTile tl_next = blockIdx.x < p.ntiles ? p.tiles[blockIdx.x] : ZTile{};
        for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
            const ZTile tl = tl_next;
            if (t + (int)gridDim.x < p.ntiles) tl_next = p.tiles[t + gridDim.x];
            const int4 W = p.wxyz[tl.w];
            const int gt = tl.mrow / ZT_BM, nch = p.nchunk[gt];
            const int slot = p.kslot[tl.k];
            const int2 *so = p.segoff + (size_t)gt * p.nsegp_max;
            const int *runs = p.runs + (size_t)gt * (p.nsegp_max / KSEG);
            // a segment starts at X = W_x + x - tlo_x, Y likewise, and T z index
            // Zs = W_z - tlo_z + z0: copy Zs mod 4, z block Zs / 4 -- inside the
            // box by construction
            const int bxy = (W.x - p.tlo0) * p.td1 + (W.y - p.tlo1);
            const int bz = W.z - p.tlo2;
            bool stop = false;
            int ri_next = nch > 0 ? runs[0] : 0;
            int2 sg_next = (nch > 0 && lane < KSEG) ? so[lane] : make_int2(0, 0);
            for (int c = 0; c < nch; ++c) {
                const int ri = ri_next, live = ri >> 8, starts = ri & 0xff;
                const int2 sg = sg_next;
                if (c + 1 < nch) {
                    ri_next = runs[c + 1];
                    if (lane < KSEG) sg_next = so[(c + 1) * KSEG + lane];
                }
                int ok = 1;
                if (lane == 0) {
                    ok = mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, p.err, kDevTimeoutTma) ? 1 : 0;
                    if (ok) mbar_expect_tx(&full_bar[s], NPL * ZT_A_PLANE + live * SEG4);
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) { stop = true; break; }
                unsigned char *st = stages + (size_t)s * STAGE;
                if (lane < NPL)
                    tma_load_2d(saddr(st + lane * ZT_A_PLANE), &tmA, &full_bar[s], c * KC, lane * p.Rpad + tl.mrow);
                if (lane < live && ((starts >> lane) & 1)) {
                    const int rest = starts >> (lane + 1);
                    const int len = rest ? __ffs(rest) : live - lane;   // segments up to the next run
                    const int Zs = bz + sg.y;
                    const int cp = Zs & (ZT_NCOPY - 1);
                    const long long cell =
                        (((long long)cp * p.nslot + slot) * ((long long)p.td0 * p.td1) + bxy + sg.x) * p.nzb + Zs / ZT_SEGZ;
                    bulk_load(saddr(st + NPL * ZT_A_PLANE + lane * SEG4), tq + (cell * p.nblk + tl.nblk) * SEG4,
                              (uint32_t)(len * SEG4), &full_bar[s]);
                }
                ++issued;
                if (++s == ZT_STAGES) { s = 0; ph ^= 1; }
            }
            if (stop) break;
        }
        __syncwarp();
        if (lane == 0 && abort_flag) {
            for (int i = 0; i < ZT_STAGES && i < issued; ++i) mbar_drain(&full_bar[i], 0), mbar_drain(&full_bar[i], 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, eph = 0;
            // A slice a times the B slices b = 0 .. 3 - a, stacked in N (the B planes
            // are contiguous), lands in the class columns (a + b) N: five MMAs per
            // K step cover the ten slice products
            constexpr bool three = 3 * N <= 256;           // a1 x (b0, b1, b2) in one MMA
            constexpr uint32_t id1 = idesc_bf16(ZT_BM, N), id2 = idesc_bf16(ZT_BM, 2 * N),
                               id3 = idesc_bf16(ZT_BM, three ? 3 * N : N);
            static_assert(2 * N <= 256 && (N % 16) == 0, "stacked B planes exceed the MMA width");
            bool ok = true;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
                const ZTile tm0 = p.tiles[t];
                const int nchunk = p.nchunk[tm0.mrow / ZT_BM];
                for (int g0 = 0; g0 < nchunk && ok; g0 += ZT_GROUP) {
                    if (!mbar_wait(&tempty_bar, eph ^ 1, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                    tc_fence_after();
                    for (int c = g0; c < min(nchunk, g0 + ZT_GROUP); ++c) {
                        if (!mbar_wait(&full_bar[s], ph, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                        tc_fence_after();
                        unsigned char *st = stages + (size_t)s * STAGE;
                        const uint32_t a0 = saddr(st), b0 = saddr(st + NPL * ZT_A_PLANE);
                        const bool first = c == g0;
#pragma unroll
                        for (int ks = 0; ks < KSEG / 2; ++ks) {
                            // K step ks: segments 2 ks and 2 ks + 1 (B planes from plane b on)
                            auto dsc = [](uint32_t a) { return KSEG == 8 ? desc_sw128(a) : desc_sw64(a); };
                            const uint64_t d0 = dsc(a0) + 2 * ks;
                            const uint64_t d1 = dsc(a0 + ZT_A_PLANE) + 2 * ks;
                            const uint64_t d2 = dsc(a0 + 2 * ZT_A_PLANE) + 2 * ks;
                            const uint64_t d3 = dsc(a0 + 3 * ZT_A_PLANE) + 2 * ks;
                            const uint64_t e0 = desc_ns(b0 + 2 * ks * SEG4, SEG4, 128);
                            const uint64_t e2 = desc_ns(b0 + 2 * ks * SEG4 + 2 * SEGB, SEG4, 128);
                            const uint32_t acc = (first && ks == 0) ? 0u : 1u;   // the two a = 0 MMAs set all classes
                            umma_bf16(tmem, d0, e0, id2, acc);                 // classes 0, 1
                            umma_bf16(tmem + 2 * N, d0, e2, id2, acc);         // classes 2, 3
                            if (three) {
                                umma_bf16(tmem + N, d1, e0, id3, 1u);          // classes 1, 2, 3
                            } else {
                                umma_bf16(tmem + N, d1, e0, id2, 1u);          // classes 1, 2
                                umma_bf16(tmem + 3 * N, d1, e2, id1, 1u);      // class 3
                            }
                            umma_bf16(tmem + 2 * N, d2, e0, id2, 1u);          // classes 2, 3
                            umma_bf16(tmem + 3 * N, d3, e0, id1, 1u);          // class 3
                        }
                        umma_commit(&empty_bar[s]);
                        if (++s == ZT_STAGES) { s = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    umma_commit(&tfull_bar);
                    eph ^= 1;
                }
            }
            umma_drain(&mma_done);
        }
    }
    } else {
        if constexpr (zt_split(NB)) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(ZT_REG_EPI));
        // epilogue warp (quarter, cs): TMEM lanes of its quarter, bands
        // [cs NB/2, (cs + 1) NB/2) of the block, real and imaginary columns of each
        constexpr int NH = NB / 2;                     // a multiple of 4
        const int e = warp - 4;
        const int quarter = warp % 4, cs = e / 4;
        uint32_t eph = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            const ZTile tl = p.tiles[t];
            const int4 W = p.wxyz[tl.w];
            const int ngroups = (p.nchunk[tl.mrow / ZT_BM] + ZT_GROUP - 1) / ZT_GROUP;   // same grouping as the MMA warp
            // everything the output of this row needs, fetched now so that the
            // dependent loads overlap the first K group instead of following it:
            // the output row g, the first column and the live bands, the scales
            int g = -1, nlive = 0, ea = 0;
            long long col = 0;
            {
                // the band exponents of this warp's bands (the same for every row of
                // the tile: one k) go to shared memory, one per lane; the row's own
                // exponent stays in a register
                const int n0 = tl.nblk * NB + cs * NH;
                __syncwarp();
                s_eT[e][lane] = (lane < NH && n0 + lane < p.nbmax) ? p.eT[(size_t)tl.k * p.nbmax + n0 + lane] : 0;
                __syncwarp();
                const int r = tl.mrow + quarter * 32 + lane;
                if (r < p.R) {
                    const int kp = p.rowk[r], m = p.rowm[r];
                    const ZPairInfo pi = p.pinfo[(size_t)tl.k * p.nk + kp];
                    if (pi.pair >= 0) {
                        const PairDesc pr = p.pairs[pi.pair];
                        const int Gx = W.x + pi.g0x - p.ax0, Gy = W.y + pi.g0y - p.ay0, Gz = W.z + pi.g0z - p.az0;
                        if (Gx >= 0 && Gx < p.ad0 && Gy >= 0 && Gy < p.ad1 && Gz >= 0 && Gz < p.ad2)
                            g = p.gtab[(((size_t)pr.qslot * p.ad0 + Gx) * p.ad1 + Gy) * p.ad2 + Gz];
                        nlive = min(NH, pr.nb - n0);
                        col = pr.col0 + (long long)m * pr.nb + n0;
                        ea = p.aexp[r] - 16;
                    }
                }
            }
            uint64_t hr[NH / 2], lr[NH / 2], hm[NH / 2], lm[NH / 2];   // packed pairs of columns
#pragma unroll
            for (int j = 0; j < NH / 2; ++j) { hr[j] = 0; lr[j] = 0; hm[j] = 0; lm[j] = 0; }
            for (int g = 0; g < ngroups; ++g) {
                if (!mbar_wait(&tfull_bar, eph, &abort_flag, p.err, kDevTimeoutEpi)) { ok = false; break; }
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + cs * NH;
#pragma unroll
                for (int c0 = 0; c0 < NH; c0 += 4) {
                    uint32_t a0[4], a1[4], a2[4], a3[4], b0[4], b1[4], b2[4], b3[4];
                    tmem_ld4(tb + 0 * N + c0, a0);
                    tmem_ld4(tb + 1 * N + c0, a1);
                    tmem_ld4(tb + 2 * N + c0, a2);
                    tmem_ld4(tb + 3 * N + c0, a3);
                    tmem_ld4(tb + 0 * N + NB + c0, b0);
                    tmem_ld4(tb + 1 * N + NB + c0, b1);
                    tmem_ld4(tb + 2 * N + NB + c0, b2);
                    tmem_ld4(tb + 3 * N + NB + c0, b3);
                    tmem_wait_ld();
                    if (c0 + 4 >= NH) {   // everything read: hand the accumulators back to the MMA warp
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty_bar);
                    }
#pragma unroll
                    for (int j = 0; j < 4; j += 2) {
                        class_accumulate2(f2_pack(a0[j], a0[j + 1]), f2_pack(a1[j], a1[j + 1]), f2_pack(a2[j], a2[j + 1]),
                                          f2_pack(a3[j], a3[j + 1]), hr[(c0 + j) / 2], lr[(c0 + j) / 2]);
                        class_accumulate2(f2_pack(b0[j], b0[j + 1]), f2_pack(b1[j], b1[j + 1]), f2_pack(b2[j], b2[j + 1]),
                                          f2_pack(b3[j], b3[j + 1]), hm[(c0 + j) / 2], lm[(c0 + j) / 2]);
                    }
                }
                eph ^= 1;
            }
            if (!ok) break;
            if (g >= 0) {
                // G-major: this row's bands are consecutive columns of row g, so the
                // thread's stores fill whole sectors (the transpose into Z follows)
                double2 *out = p.ZI + (size_t)g * p.NCi + col;
#pragma unroll
                for (int jj = 0; jj < NH; ++jj) {
                    if (jj < nlive) {
                        const float2 h1 = f2_unpack(hr[jj / 2]), l1 = f2_unpack(lr[jj / 2]);
                        const float2 h2 = f2_unpack(hm[jj / 2]), l2 = f2_unpack(lm[jj / 2]);
                        const bool odd = jj & 1;
                        // Omega^{-1/2} is in the C slices; the conversion runs on the integer
                        // units (measured faster here than the one-FP64-add form)
                        double2 v;
                        const int ex = ea + s_eT[e][jj];
                        v.x = f32pair_to_f64_int(odd ? h1.y : h1.x, odd ? l1.y : l1.x, ex);
                        v.y = f32pair_to_f64_int(odd ? h2.y : h2.x, odd ? l2.y : l2.x, ex);
                        __stcs(out + jj, v);   // streaming: keep the operands in L2
                    }
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

// Z[col][nmt + g] = ZI[g][col] for the interstitial rows g < nipw(q) of every
// column of every q of the batch: 32 x 32 tiles through shared memory, reads
// along the columns of ZI and writes along the rows of Z, both coalesced.
__global__ void __launch_bounds__(256) ipw_transpose_kernel(const double2 *__restrict__ ZI, long long NCi,
                                                            double2 *__restrict__ Z, long long RSc, int nmt,
                                                            const QDesc *__restrict__ qd) {
    __shared__ double2 tile[32][33];
    const QDesc q = qd[blockIdx.z];
    const long long c0 = (long long)blockIdx.x * 32;
    const int g0 = blockIdx.y * 32;
    if (c0 >= q.ncols || g0 >= q.nipw) return;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int g = g0 + ty + 8 * i;
        const long long c = c0 + tx;
        if (g < q.nipw && c < q.ncols) tile[ty + 8 * i][tx] = ZI[(size_t)g * NCi + q.colbase + c];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long c = c0 + ty + 8 * i;
        const int g = g0 + tx;
        if (g < q.nipw && c < q.ncols) Z[(size_t)(q.colbase + c) * RSc + nmt + g] = tile[tx][ty + 8 * i];
    }
}

// band block: a multiple of 8 (the output width 2 NB is a multiple of 16),
// at most 40 (two pipeline stages in shared memory), fewest padded bands
int pick_nb(int nb_max) {
    int best = 8, best_tot = 1 << 30;
    for (int nb = 8; nb <= 40; nb += 8) {
        int tot = (nb_max + nb - 1) / nb * nb;
        if (tot < best_tot || (tot == best_tot && nb > best)) { best = nb; best_tot = tot; }
    }
    return best;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side, per build: the rows (k', m) in Morton order of k', the segment
// grid of every row tile, the C slices and the band exponents of T.
int zipw_tc_plan_build(hfx_ctx *ctx, const std::vector<int> &kset, int nb_max, const int tlo[3], const int tdim[3],
                       int nb_tile, HostArena &tab, ZipwBuild &zb) {
    zb = ZipwBuild();
    const int nk = ctx->nk;
    // ---- G1 lines (x, y) with their z ranges over every k' plane-wave list
    int gmin[3] = {1 << 29, 1 << 29, 1 << 29}, gmax[3] = {-(1 << 29), -(1 << 29), -(1 << 29)};
    for (auto &k : ctx->kp)
        for (size_t i = 0; i < k.G.size(); ++i) {
            int x = i % 3;
            gmin[x] = std::min(gmin[x], k.G[i]);
            gmax[x] = std::max(gmax[x], k.G[i]);
        }
    if (gmin[0] > gmax[0]) return HFX_OK;
    const int Bx = gmax[0] - gmin[0] + 1, By = gmax[1] - gmin[1] + 1;
    std::vector<int> zlo((size_t)Bx * By, 1 << 29), zhi((size_t)Bx * By, -(1 << 29));
    for (auto &k : ctx->kp)
        for (size_t i = 0; i + 2 < k.G.size(); i += 3) {
            size_t b = (size_t)(k.G[i] - gmin[0]) * By + (k.G[i + 1] - gmin[1]);
            zlo[b] = std::min(zlo[b], k.G[i + 2]);
            zhi[b] = std::max(zhi[b], k.G[i + 2]);
        }
    std::vector<int> line_of((size_t)Bx * By, -1), lx, ly, lzlo;
    for (int x = 0; x < Bx; ++x)
        for (int y = 0; y < By; ++y) {
            size_t b = (size_t)x * By + y;
            if (zlo[b] > zhi[b]) continue;
            line_of[b] = (int)lx.size();
            lx.push_back(gmin[0] + x);
            ly.push_back(gmin[1] + y);
            lzlo.push_back(zlo[b]);
        }
    const int nL = (int)lx.size();
    // ---- rows (k', m): k' in Morton order of their mesh indices, so that a
    // 128-row tile holds a compact block of the mesh (overlapping spheres)
    const int *Mh = ctx->sys.mesh;
    auto morton = [&](int ik) {
        const int j[3] = {ik / (Mh[1] * Mh[2]), (ik / Mh[2]) % Mh[1], ik % Mh[2]};
        unsigned long long code = 0;
        for (int bit = 0; bit < 20; ++bit)
            for (int x = 0; x < 3; ++x) code |= (unsigned long long)((j[x] >> bit) & 1) << (3 * bit + 2 - x);
        return code;
    };
    std::vector<int> korder(nk);
    for (int i = 0; i < nk; ++i) korder[i] = i;
    std::stable_sort(korder.begin(), korder.end(), [&](int a, int b2) { return morton(a) < morton(b2); });
    std::vector<int> rowk, rowm;
    zb.rowbase.assign(nk, -1);
    for (int kp : korder) {
        zb.rowbase[kp] = (int)rowk.size();
        for (int m = 0; m < ctx->kp[kp].nom; ++m) { rowk.push_back(kp); rowm.push_back(m); }
    }
    const int R = (int)rowk.size();
    if (R == 0) return HFX_OK;
    const int Rpad = (R + ZT_BM - 1) / ZT_BM * ZT_BM;
    const int nmtile = Rpad / ZT_BM;
    std::vector<std::vector<int>> tile_k(nmtile);
    for (int r = 0; r < R; ++r)
        if (tile_k[r / ZT_BM].empty() || tile_k[r / ZT_BM].back() != rowk[r]) tile_k[r / ZT_BM].push_back(rowk[r]);
    // segment grid per row tile: the lines of the tile's spheres, each cut
    // into segments of ZT_SEGZ z values from its lowest z
    std::vector<int> segstart((size_t)nmtile * nL, 0), segz0((size_t)nmtile * nL, 0), nseg(nmtile);
    std::vector<std::vector<int4>> segs(nmtile);
    std::vector<int> tzlo(nL), tzhi(nL);
    for (int t = 0; t < nmtile; ++t) {
        std::fill(tzlo.begin(), tzlo.end(), 1 << 29);
        std::fill(tzhi.begin(), tzhi.end(), -(1 << 29));
        for (int kp : tile_k[t]) {
            const std::vector<int> &G = ctx->kp[kp].G;
            for (size_t i = 0; i + 2 < G.size(); i += 3) {
                int l = line_of[(size_t)(G[i] - gmin[0]) * By + (G[i + 1] - gmin[1])];
                tzlo[l] = std::min(tzlo[l], G[i + 2]);
                tzhi[l] = std::max(tzhi[l], G[i + 2]);
            }
        }
        for (int l = 0; l < nL; ++l) {
            if (tzlo[l] > tzhi[l]) continue;
            segstart[(size_t)t * nL + l] = (int)segs[t].size();
            segz0[(size_t)t * nL + l] = tzlo[l];
            for (int z = tzlo[l]; z <= tzhi[l]; z += ZT_SEGZ) segs[t].push_back(make_int4(lx[l], ly[l], z, 0));
        }
        if (segs[t].empty()) segs[t].push_back(make_int4(lx[0], ly[0], lzlo[0], 0));
        nseg[t] = (int)segs[t].size();
    }
    int nsegp_max = 0;
    for (int t = 0; t < nmtile; ++t) nsegp_max = std::max(nsegp_max, (nseg[t] + 7) / 8 * 8);
    const int Kp = nsegp_max * 8;   // K values of an A row: 8 per segment
    const int nzb = (tdim[2] + ZT_SEGZ - 1) / ZT_SEGZ;
    const int NBt = zipw_tc_valid_nb(nb_tile) ? nb_tile : pick_nb(nb_max);
    const int nblk = (nb_max + NBt - 1) / NBt;
    const int KSEG = zt_kseg(NBt);   // segments per K chunk of the kernel instance
    std::vector<int2> segtab((size_t)nmtile * nsegp_max);
    std::vector<int> nchunk(nmtile);
    for (int t = 0; t < nmtile; ++t) {
        nchunk[t] = (nseg[t] + KSEG - 1) / KSEG;
        for (int s2 = 0; s2 < nsegp_max; ++s2) {
            const int4 sg = s2 < nseg[t] ? segs[t][s2] : segs[t][0];   // padding: any valid block
            segtab[(size_t)t * nsegp_max + s2] = make_int2(sg.x * tdim[1] + sg.y, sg.z);
        }
    }
    // bulk-copy runs per K chunk: consecutive segments of one line are
    // consecutive z blocks of T, contiguous for a single band block
    std::vector<int> runs((size_t)nmtile * (nsegp_max / KSEG), 0);
    for (int t = 0; t < nmtile; ++t)
        for (int c = 0; c < nsegp_max / KSEG; ++c) {
            const int live = std::max(0, std::min(KSEG, nseg[t] - KSEG * c));
            int starts = 0;
            for (int j = 0; j < live; ++j) {
                const int s2 = KSEG * c + j;
                const bool cont = j > 0 && nblk == 1 && segs[t][s2].x == segs[t][s2 - 1].x &&
                                  segs[t][s2].y == segs[t][s2 - 1].y && segs[t][s2].z == segs[t][s2 - 1].z + ZT_SEGZ;
                if (!cont) starts |= 1 << j;
            }
            runs[(size_t)t * (nsegp_max / KSEG) + c] = starts | (live << 8);
        }
    // extent of every segment start, for the per-batch box check
    zb.sx0 = zb.sy0 = zb.sz0 = 1 << 29;
    zb.sx1 = zb.sy1 = zb.sz1 = -(1 << 29);
    for (int t = 0; t < nmtile; ++t)
        for (const int4 &sg : segs[t]) {
            zb.sx0 = std::min(zb.sx0, sg.x); zb.sx1 = std::max(zb.sx1, sg.x);
            zb.sy0 = std::min(zb.sy0, sg.y); zb.sy1 = std::max(zb.sy1, sg.y);
            zb.sz0 = std::min(zb.sz0, sg.z); zb.sz1 = std::max(zb.sz1, sg.z);
        }
    std::vector<int> kall(nk, -1);
    for (int ik : kset) kall[ik] = 0;
    zb.o_rowk = tab.put(rowk);
    zb.o_rowm = tab.put(rowm);
    zb.o_line = tab.put(line_of);
    zb.o_sst = tab.put(segstart);
    zb.o_sz0 = tab.put(segz0);
    zb.o_seg = tab.put(segtab);
    zb.o_nch = tab.put(nchunk);
    zb.o_runs = tab.put(runs);
    zb.o_kall = tab.put(kall);
    // device scratch of the build: C slices, their row exponents, band exponents of T
    Layout lay;
    zb.a_elems = (size_t)NPL * Rpad * Kp;
    zb.s_a = lay.place(zb.a_elems * 2);
    zb.s_aexp = lay.place((size_t)Rpad * 4);
    zb.s_eT = lay.place((size_t)nk * nb_max * 4);
    zb.scratch_bytes = lay.off;
    zb.R = R; zb.Rpad = Rpad; zb.nmtile = nmtile; zb.nL = nL; zb.gx0 = gmin[0]; zb.gy0 = gmin[1]; zb.By = By;
    zb.nsegp_max = nsegp_max; zb.Kp = Kp; zb.NBt = NBt; zb.nblk = nblk; zb.nbpad = nblk * NBt; zb.nzb = nzb;
    zb.nb_max = nb_max;
    for (int x = 0; x < 3; ++x) { zb.tlo[x] = tlo[x]; zb.tdim[x] = tdim[x]; }
    zb.tq_bytes_per_slot = (size_t)ZT_NCOPY * tdim[0] * tdim[1] * nzb * NPL * 2 * zb.nbpad * 8 * 2;
    zb.ok = true;
    return HFX_OK;
}

// Host side, per batch: the shifts W = G - G0 every row tile needs for each k
// of the batch, the aux lookup over the batch's q, and the tiles.
int zipw_tc_plan_batch(hfx_ctx *ctx, const ZipwBuild &zb, const std::vector<int> &qs, const std::vector<PairDesc> &pairs,
                       HostArena &tab, ZipwBatch &bt) {
    bt = ZipwBatch();
    if (!zb.ok) return HFX_OK;
    const int nk = ctx->nk, nmtile = zb.nmtile;
    // ---- aux lookup tables over the batch's q
    int amin[3] = {1 << 29, 1 << 29, 1 << 29}, amax[3] = {-(1 << 29), -(1 << 29), -(1 << 29)};
    for (int iq : qs)
        for (size_t i = 0; i < ctx->qp[iq].G.size(); ++i) {
            int x = i % 3;
            amin[x] = std::min(amin[x], ctx->qp[iq].G[i]);
            amax[x] = std::max(amax[x], ctx->qp[iq].G[i]);
        }
    int ad[3];
    for (int x = 0; x < 3; ++x) {
        if (amin[x] > amax[x]) amin[x] = amax[x] = 0;
        ad[x] = amax[x] - amin[x] + 1;
    }
    const int nq = (int)qs.size();
    std::vector<int> gtab((size_t)nq * ad[0] * ad[1] * ad[2], -1);
    for (int s = 0; s < nq; ++s) {
        const std::vector<int> &G = ctx->qp[qs[s]].G;
        for (size_t g = 0; g < G.size() / 3; ++g)
            gtab[(((size_t)s * ad[0] + (G[3 * g] - amin[0])) * ad[1] + (G[3 * g + 1] - amin[1])) * ad[2] + (G[3 * g + 2] - amin[2])] = (int)g;
    }
    // ---- pair info (k, k') and the shift lists / tiles per k of the batch
    std::vector<ZPairInfo> pinfo((size_t)nk * nk, ZPairInfo{-1, 0, 0, 0});
    std::vector<int> bks;     // k of the batch in first-appearance order
    std::vector<int> kslot(nk, -1);
    for (int i = 0; i < (int)pairs.size(); ++i) {
        const PairDesc &pr = pairs[i];
        pinfo[(size_t)pr.ik * nk + pr.ikp] = ZPairInfo{i, pr.g0[0], pr.g0[1], pr.g0[2]};
        if (kslot[pr.ik] < 0) { kslot[pr.ik] = (int)bks.size(); bks.push_back(pr.ik); }
    }
    // W = G - G0 lies in [amin, amax + 1]
    const int wd[3] = {ad[0] + 1, ad[1] + 1, ad[2] + 1};
    const size_t wvol = (size_t)wd[0] * wd[1] * wd[2];
    std::vector<int4> wxyz;
    std::vector<ZTile> tiles;
    std::vector<unsigned char> need;
    for (int ik : bks) {
        need.assign(wvol * nmtile, 0);
        for (const PairDesc &pr : pairs) {
            if (pr.ik != ik || pr.no == 0) continue;
            const std::vector<int> &G = ctx->qp[pr.iq].G;
            const int t0 = zb.rowbase[pr.ikp] / ZT_BM, t1 = (zb.rowbase[pr.ikp] + pr.no - 1) / ZT_BM;
            for (size_t g = 0; g < G.size() / 3; ++g) {
                int w0 = G[3 * g] - pr.g0[0] - amin[0], w1 = G[3 * g + 1] - pr.g0[1] - amin[1], w2 = G[3 * g + 2] - pr.g0[2] - amin[2];
                size_t wi = ((size_t)w0 * wd[1] + w1) * wd[2] + w2;
                for (int t = t0; t <= t1; ++t) need[wi * nmtile + t] = 1;
            }
        }
        for (size_t wi = 0; wi < wvol; ++wi) {
            bool any = false;
            for (int t = 0; t < nmtile; ++t) any |= need[wi * nmtile + t] != 0;
            if (!any) continue;
            const int widx = (int)wxyz.size();
            const int w2 = (int)(wi % wd[2]), w1 = (int)((wi / wd[2]) % wd[1]), w0 = (int)(wi / ((size_t)wd[1] * wd[2]));
            wxyz.push_back(make_int4(w0 + amin[0], w1 + amin[1], w2 + amin[2], 0));
            for (int t = 0; t < nmtile; ++t)
                if (need[wi * nmtile + t])
                    for (int b = 0; b < zb.nblk; ++b) tiles.push_back(ZTile{ik, widx, t * ZT_BM, b});
        }
    }
    if (tiles.empty()) return HFX_OK;
    // every B segment of every tile must be one whole z block inside the sliced T box
    for (const int4 &W : wxyz) {
        const int Z0 = W.z + zb.sz0 - zb.tlo[2], Z1 = W.z + zb.sz1 - zb.tlo[2];
        if (W.x + zb.sx0 - zb.tlo[0] < 0 || W.x + zb.sx1 - zb.tlo[0] >= zb.tdim[0] || W.y + zb.sy0 - zb.tlo[1] < 0 ||
            W.y + zb.sy1 - zb.tlo[1] >= zb.tdim[1] || Z0 < 0 || Z1 / ZT_SEGZ >= zb.nzb)
            return set_err(ctx, HFX_EUNSUPPORTED, "interstitial segment outside the step-function box");
    }
    if (tiles.size() > (size_t)0x7fffffff) return set_err(ctx, HFX_EUNSUPPORTED, "interstitial tile list too long");
    bt.o_gtab = tab.put(gtab);
    bt.o_pinfo = tab.put(pinfo);
    bt.o_w = tab.put(wxyz);
    bt.o_tiles = tab.put(tiles);
    bt.o_kslot = tab.put(kslot);
    bt.ntiles = (int)tiles.size();
    bt.nslot = (int)bks.size();
    for (int x = 0; x < 3; ++x) { bt.amin[x] = amin[x]; bt.ad[x] = ad[x]; }
    bt.tq_bytes = zb.tq_bytes_per_slot * bt.nslot;
    bt.ok = true;
    return HFX_OK;
}

// Per build: C slices of every row (k', m) and the band exponents of T_k.
int zipw_tc_run_build(hfx_ctx *ctx, const ZipwBuild &zb, const char *dtab, char *dscr, const double2 *const *d_ck,
                      const int *const *d_Gk, const int *d_npw, const double2 *const *d_Tk, const int *d_nb) {
    if (!zb.ok) return HFX_OK;
    cudaStream_t st = ctx->stream;
    __nv_bfloat16 *A = reinterpret_cast<__nv_bfloat16 *>(dscr + zb.s_a);
    int *aexp = reinterpret_cast<int *>(dscr + zb.s_aexp), *eT = reinterpret_cast<int *>(dscr + zb.s_eT);
    cudaMemsetAsync(aexp, 0, (size_t)zb.Rpad * 4, st);
    cudaMemsetAsync(A, 0, zb.a_elems * 2, st);
    c_slices_kernel<<<zb.R, 256, 0, st>>>(d_ck, d_Gk, d_npw, reinterpret_cast<const int *>(dtab + zb.o_rowk),
                                          reinterpret_cast<const int *>(dtab + zb.o_rowm),
                                          reinterpret_cast<const int *>(dtab + zb.o_line), zb.gx0, zb.gy0, zb.By, zb.nL,
                                          reinterpret_cast<const int *>(dtab + zb.o_sst),
                                          reinterpret_cast<const int *>(dtab + zb.o_sz0), zb.Kp, zb.Rpad,
                                          1.0 / sqrt(ctx->omega), A, aexp);
    t_exp_kernel<<<dim3(zb.nb_max, ctx->nk), 256, 0, st>>>(d_Tk, d_nb, zb.tdim[0], zb.tdim[1], zb.tdim[2], zb.nb_max,
                                                           reinterpret_cast<const int *>(dtab + zb.o_kall), eT);
    return cuda_check(ctx, cudaGetLastError(), "zipw slices");
}

int zipw_tc_valid_nb(int nb) { return nb >= 8 && nb <= 64 && nb % 8 == 0; }

// Per batch: T slices of the batch's k and the GEMM.
int zipw_tc_run_batch(hfx_ctx *ctx, const ZipwBuild &zb, const ZipwBatch &bt, const char *dtab, const char *dscr,
                      __nv_bfloat16 *dTq, const PairDesc *d_pairs, const double2 *const *d_Tk, const int *d_nb,
                      double2 *d_Z, long long RSc, double2 *d_ZI, long long NCi, const QDesc *d_qd, int nq,
                      long long maxcols, int max_nipw, cudaEvent_t ev0, cudaEvent_t ev1, int *nlaunch) {
    if (!zb.ok || !bt.ok) return HFX_OK;
    cudaStream_t st = ctx->stream;
    int rc;
    const int *kslot = reinterpret_cast<const int *>(dtab + bt.o_kslot);
    {
        const long long nthreads = (long long)zb.tdim[0] * zb.tdim[1] * zb.nzb * zb.nbpad;
        t_slices_kernel<<<dim3((unsigned)((nthreads + 255) / 256), ctx->nk), 256, 0, st>>>(
            d_Tk, d_nb, zb.tdim[0], zb.tdim[1], zb.tdim[2], zb.nzb, zb.NBt, zb.nblk, zb.nb_max, bt.nslot, kslot,
            reinterpret_cast<const int *>(dscr + zb.s_eT), dTq);
    }
    if ((rc = cuda_check(ctx, cudaGetLastError(), "zipw T slices"))) return rc;
    CUtensorMap mA;
    const int KSEG = zt_kseg(zb.NBt), KC = 8 * KSEG;
    if ((rc = make_map_2d_sw(ctx, &mA, dscr + zb.s_a, (long long)NPL * zb.Rpad, zb.Kp, ZT_BM, KC, 2 * KC))) return rc;
    ZParams p;
    p.tiles = reinterpret_cast<const ZTile *>(dtab + bt.o_tiles);
    p.ntiles = bt.ntiles;
    p.wxyz = reinterpret_cast<const int4 *>(dtab + bt.o_w);
    p.pinfo = reinterpret_cast<const ZPairInfo *>(dtab + bt.o_pinfo);
    p.pairs = d_pairs;
    p.gtab = reinterpret_cast<const int *>(dtab + bt.o_gtab);
    p.ax0 = bt.amin[0]; p.ay0 = bt.amin[1]; p.az0 = bt.amin[2];
    p.ad0 = bt.ad[0]; p.ad1 = bt.ad[1]; p.ad2 = bt.ad[2];
    p.rowk = reinterpret_cast<const int *>(dtab + zb.o_rowk);
    p.rowm = reinterpret_cast<const int *>(dtab + zb.o_rowm);
    p.aexp = reinterpret_cast<const int *>(dscr + zb.s_aexp);
    p.eT = reinterpret_cast<const int *>(dscr + zb.s_eT);
    p.kslot = kslot;
    p.segoff = reinterpret_cast<const int2 *>(dtab + zb.o_seg);
    p.nsegp_max = zb.nsegp_max;
    p.nchunk = reinterpret_cast<const int *>(dtab + zb.o_nch);
    p.runs = reinterpret_cast<const int *>(dtab + zb.o_runs);
    p.Tq = dTq;
    p.td0 = zb.tdim[0];
    p.td1 = zb.tdim[1];
    p.nzb = zb.nzb;
    p.nblk = zb.nblk;
    p.nslot = bt.nslot;
    p.ZI = d_ZI;
    p.NCi = NCi;
    p.nmt = ctx->nmt;
    p.nk = ctx->nk;
    p.R = zb.R;
    p.Rpad = zb.Rpad;
    p.nbmax = zb.nb_max;
    p.tlo0 = zb.tlo[0]; p.tlo1 = zb.tlo[1]; p.tlo2 = zb.tlo[2];
    p.rs = 1.0 / sqrt(ctx->omega);
    p.err = ctx->d_err;
    const int grid = std::min<int>(num_sms(), p.ntiles);
    // the whole opt-in shared memory: the pipeline stages plus a guard region
    // past the last stage that no descriptor of the B operand can reach beyond
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int rc_launch = HFX_OK;
    auto go = [&](auto kern, int nb) {
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, kern);
        if (zt_split(nb) && fa.numRegs < ZT_REG_LAUNCH) {
            // the register split assumes this launch allocation
            rc_launch = set_err(ctx, HFX_EUNSUPPORTED, "zipw kernel compiled with fewer registers than its warpgroup split needs");
            return;
        }
        const size_t stage = (size_t)NPL * 128 * KC * 2 + (size_t)KSEG * NPL * 2 * nb * 16;
        size_t smem = std::max<size_t>((size_t)zt_stages(KSEG) * stage + 1024, (size_t)smem_max - fa.sharedSizeBytes);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (ev0) record_event(ev0, st);
        kern<<<grid, ZT_THREADS, smem, st>>>(mA, p);
        if (ev1) record_event(ev1, st);
    };
    switch (zb.NBt) {
    case 8: go(zipw_tc_kernel<8>, 8); break;
    case 16: go(zipw_tc_kernel<16>, 16); break;
    case 24: go(zipw_tc_kernel<24>, 24); break;
    case 32: go(zipw_tc_kernel<32>, 32); break;
    case 40: go(zipw_tc_kernel<40>, 40); break;
    case 48: go(zipw_tc_kernel<48>, 48); break;
    case 56: go(zipw_tc_kernel<56>, 56); break;
    default: go(zipw_tc_kernel<64>, 64); break;
    }
    if (rc_launch) return rc_launch;
    if ((rc = cuda_check(ctx, cudaGetLastError(), "zipw tensor-core kernel"))) return rc;
    if (nq > 0 && maxcols > 0 && max_nipw > 0) {
        const dim3 tg((unsigned)((maxcols + 31) / 32), (unsigned)((max_nipw + 31) / 32), (unsigned)nq);
        ipw_transpose_kernel<<<tg, 256, 0, st>>>(d_ZI, NCi, d_Z, RSc, ctx->nmt, d_qd);
    }
    if (nlaunch) *nlaunch += 3;
    return cuda_check(ctx, cudaGetLastError(), "interstitial transpose");
}

}  // namespace hfx
