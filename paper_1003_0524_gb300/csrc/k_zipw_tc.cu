// k_zipw_tc.cu -- interstitial projections on the tensor cores.
//
//   Z_kq[G, m, n] = Omega^{-1/2} sum_{G1 in k'} conj(c_{G1}(m, k')) T_n(G + G1 - G0)   (Sec. III.B)
//
// For a fixed k and a fixed shift W = G - G0, every (k', m) row of every pair
// (k, q) that needs this W is one row of a GEMM
//   Z[(k', m), n] = sum_{G1} C[(k', m), G1] T_k[n](W + G1),   C = conj(c),
// whose reduction index G1 runs over a common box organised in (x, y) lines
// of 16 z values.  A = C (fixed per k', loaded by 2-D TMA, 128-byte swizzle);
// B = T_k shifted by W, one TMA box of 16 z x all bands per line (32-byte
// swizzle), read from eight z-shifted copies so that every TMA start
// coordinate is 16-byte aligned.  Complex arithmetic uses the real embedding;
// all operands are fixed-point slices (tc_ptx.cuh) with exact class sums on
// the tensor cores and compensated combination on the CUDA cores.
#include <algorithm>
#include <string>
#include <vector>

#include "tc_ptx.cuh"

namespace hfx {

using namespace tc;

namespace {

__device__ __constant__ int kIA[NTERM] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
__device__ __constant__ int kIB[NTERM] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
__device__ __constant__ int kIW[NTERM] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};

// ------------------------------------------------------------- C slices
// One block per row r = (k', m): exponent over |Re c|, |Im c| of the row,
// then the real embedding rows Re r = [Re C | -Im C] and Im r = [Im C | Re C]
// (C = conj c) scattered onto the line layout K = line * 16 + (z - gz0).
__global__ void c_slices_kernel(const double2 *const *__restrict__ ck, const int *const *__restrict__ Gk,
                                const int *__restrict__ npw_k, const int *__restrict__ rowk, const int *__restrict__ rowm,
                                const int *__restrict__ line_of, int gx0, int gy0, int gz0, int By, int KH, int Rpad,
                                __nv_bfloat16 *__restrict__ A, int *__restrict__ aexp) {
    int r = blockIdx.x;
    int kp = rowk[r], m = rowm[r];
    int npw = npw_k[kp];
    const double2 *c = ck[kp] + (size_t)m * npw;
    const int *G = Gk[kp];
    long long W2 = 2LL * KH;                    // row length
    long long plane = 2LL * Rpad * W2;
    __shared__ double red[256];
    double mx = 0.0;
    for (int i = threadIdx.x; i < npw; i += blockDim.x) mx = fmax(mx, fmax(fabs(c[i].x), fabs(c[i].y)));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    int e = line_exp(red[0]);
    if (threadIdx.x == 0) {
        aexp[r] = e;
        aexp[Rpad + r] = e;
    }
    // the whole A buffer is zeroed before this kernel: only the plane waves are written
    for (int i = threadIdx.x; i < npw; i += blockDim.x) {
        int li = line_of[(G[3 * i] - gx0) * By + (G[3 * i + 1] - gy0)];
        long long K = (long long)li * 16 + (G[3 * i + 2] - gz0);
        double cr = c[i].x, ci = c[i].y;   // C = conj c = (cr, -ci)
        __nv_bfloat16 s[NPL];
        // Re row: [Re C | -Im C] = [cr | ci]
        slice4(cr, e, s);
        for (int p = 0; p < NPL; ++p) A[p * plane + (long long)r * W2 + K] = s[p];
        slice4(ci, e, s);
        for (int p = 0; p < NPL; ++p) A[p * plane + (long long)r * W2 + KH + K] = s[p];
        // Im row: [Im C | Re C] = [-ci | cr]
        slice4(-ci, e, s);
        for (int p = 0; p < NPL; ++p) A[p * plane + (long long)(Rpad + r) * W2 + K] = s[p];
        slice4(cr, e, s);
        for (int p = 0; p < NPL; ++p) A[p * plane + (long long)(Rpad + r) * W2 + KH + K] = s[p];
    }
}

// ------------------------------------------------------------- T slices
// Grid (n, k): exponent of band n of T_k over the box, then eight z-shifted
// copies Tp[k][s][p][ri][n][X][Y][z] = slice_p(part_ri(T_k[n](X, Y, z + s))).
__global__ void t_slices_kernel(const double2 *const *__restrict__ Tk, const int *__restrict__ nb_k, int td0, int td1,
                                int td2, int Zp, int nbmax, const int *__restrict__ kslot, __nv_bfloat16 *__restrict__ Tp,
                                int *__restrict__ eT) {
    int n = blockIdx.x, k = blockIdx.y;
    int slot = kslot[k];
    if (slot < 0 || n >= nb_k[k]) return;
    long long box = (long long)td0 * td1 * td2;
    const double2 *T = Tk[k] + (size_t)n * box;
    __shared__ double red[256];
    double mx = 0.0;
    for (long long i = threadIdx.x; i < box; i += blockDim.x) mx = fmax(mx, fmax(fabs(T[i].x), fabs(T[i].y)));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    int e = line_exp(red[0]);
    if (threadIdx.x == 0) eT[(size_t)k * nbmax + n] = e;
    long long lines = (long long)td0 * td1;
    long long bandsz = lines * Zp;
    for (long long i = threadIdx.x; i < 8 * lines * Zp; i += blockDim.x) {
        int z = (int)(i % Zp);
        long long xy = (i / Zp) % lines;
        int s = (int)(i / (Zp * lines));
        int zz = z + s;
        double2 v = (zz < td2) ? T[xy * td2 + zz] : make_double2(0.0, 0.0);
        __nv_bfloat16 sr[NPL], si[NPL];
        slice4(v.x, e, sr);
        slice4(v.y, e, si);
        for (int p = 0; p < NPL; ++p) {
            // rest index ((slot*8 + s)*4 + p)*2 + ri, then [n][X][Y][Zp]
            long long rr = (((long long)slot * 8 + s) * NPL + p) * 2;
            Tp[((rr + 0) * nbmax + n) * bandsz + xy * Zp + z] = sr[p];
            Tp[((rr + 1) * nbmax + n) * bandsz + xy * Zp + z] = si[p];
        }
    }
}

// ------------------------------------------------------------- GEMM
struct ZTile { int k, w, mrow, nblk; };

struct ZPairInfo { int pair; int g0x, g0y, g0z; };

struct ZParams {
    const ZTile *tiles;
    int ntiles;
    const int *wxyz;              // [nw][3] shifts W
    const ZPairInfo *pinfo;       // [nk][nk] by (k, k')
    const PairDesc *pairs;
    const int *gtab;              // [nq][ax][ay][az] aux index or -1
    int ax0, ay0, az0, ad0, ad1, ad2;
    const int *rowk, *rowm;       // rows of A (k', m)
    const int *aexp, *eT;         // row exponents, [k][n] band exponents
    const int *kslot;             // k -> slot of its T copies
    const int *line_x, *line_y;   // absolute G1 (x, y) of every line
    double2 *Z;
    long long RSc;
    int nmt, nk, R, Rpad, H, KH, nbmax, gz0, tlo0, tlo1, tlo2;
    double rs;                    // Omega^{-1/2}
    int *err;
};

constexpr int ZT_BM = 128;
constexpr int ZT_A_PLANE = 128 * 64 * 2;   // 16 KB
constexpr int ZT_GROUP = 4;                // 64-K chunks per exact group (256)
constexpr int ZT_STAGES = 2;
constexpr int ZT_EPI = 8;

// warp 0: TMA; warp 1: MMA; warps 2..9: epilogue (lane quarter, column half)
template <int NB>
__global__ void __launch_bounds__(64 + 32 * ZT_EPI, 1) zipw_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                      const __grid_constant__ CUtensorMap tmT, ZParams p) {
    constexpr int LINEB = NB * 32;                       // one line box: NB rows x 16 z
    constexpr int B_PLANE = 4 * LINEB;                   // four lines per chunk
    constexpr int STAGE = NPL * (ZT_A_PLANE + B_PLANE);
    constexpr int CW = NB / 2;
    extern __shared__ __align__(1024) unsigned char zt_smem[];
    uintptr_t base = (reinterpret_cast<uintptr_t>(zt_smem) + 1023) & ~(uintptr_t)1023;
    unsigned char *stages = reinterpret_cast<unsigned char *>(base);
    __shared__ uint64_t full_bar[ZT_STAGES], empty_bar[ZT_STAGES], tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ZT_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], ZT_EPI);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    uint32_t tmem = tmem_slot;
    const int nchunk = 2 * p.H;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            for (int t = blockIdx.x; t < p.ntiles && !abort_flag; t += gridDim.x) {
                ZTile tl = p.tiles[t];
                int Wx = p.wxyz[3 * tl.w], Wy = p.wxyz[3 * tl.w + 1], Wz = p.wxyz[3 * tl.w + 2];
                int zs = Wz + p.gz0 - p.tlo2;            // >= 0
                int shift = zs & 7, z0 = zs - shift;
                int slot = p.kslot[tl.k];
                bool stop = false;
                for (int c = 0; c < nchunk; ++c) {
                    if (!mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, p.err, kDevTimeoutTma)) { stop = true; break; }
                    int ri = c >= p.H;
                    int cl = ri ? c - p.H : c;
                    int ax = (ri ? p.KH : 0) + cl * 64;
                    unsigned char *st = stages + (size_t)s * STAGE;
                    mbar_expect_tx(&full_bar[s], STAGE);
                    for (int pl = 0; pl < NPL; ++pl) {
                        tma_load_2d(saddr(st + pl * ZT_A_PLANE), &tmA, &full_bar[s], ax, pl * 2 * p.Rpad + tl.mrow);
                        int rest = ((slot * 8 + shift) * NPL + pl) * 2 + ri;
                        for (int j = 0; j < 4; ++j) {
                            int li = cl * 4 + j;
                            int X = Wx + p.line_x[li] - p.tlo0, Y = Wy + p.line_y[li] - p.tlo1;
                            tma_load_5d(saddr(st + NPL * ZT_A_PLANE + pl * B_PLANE + j * LINEB), &tmT, &full_bar[s], z0, Y,
                                        X, tl.nblk * NB, rest);
                        }
                    }
                    ++issued;
                    if (++s == ZT_STAGES) { s = 0; ph ^= 1; }
                }
                if (stop) break;
            }
            if (abort_flag) {
                for (int i = 0; i < ZT_STAGES && i < issued; ++i) mbar_drain(&full_bar[i], 0), mbar_drain(&full_bar[i], 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int buf = 0;
            uint32_t buf_ph[2] = {0, 0};
            constexpr uint32_t idesc = idesc_bf16(ZT_BM, NB);
            bool ok = true;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
                for (int g0 = 0; g0 < nchunk && ok; g0 += ZT_GROUP) {
                    if (!mbar_wait(&tempty_bar[buf], buf_ph[buf] ^ 1, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                    tc_fence_after();
                    uint32_t dt = tmem + buf * (NPL * NB);
                    int started = 0;
                    for (int c = g0; c < min(nchunk, g0 + ZT_GROUP); ++c) {
                        if (!mbar_wait(&full_bar[s], ph, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                        tc_fence_after();
                        unsigned char *st = stages + (size_t)s * STAGE;
                        uint32_t a0 = saddr(st), b0 = saddr(st + NPL * ZT_A_PLANE);
                        for (int tm = 0; tm < NTERM; ++tm) {
                            int w = kIW[tm];
                            uint64_t da = desc_sw128(a0 + kIA[tm] * ZT_A_PLANE);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                uint64_t db = desc_sw32(b0 + kIB[tm] * B_PLANE + j * LINEB);
                                umma_bf16(dt + w * NB, da + 2 * j, db, idesc, ((started >> w) & 1) ? 1u : 0u);
                                started |= 1 << w;
                            }
                        }
                        umma_commit(&empty_bar[s]);
                        if (++s == ZT_STAGES) { s = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    umma_commit(&tfull_bar[buf]);
                    buf_ph[buf] ^= 1;
                    buf ^= 1;
                }
            }
        }
    } else {
        int e = warp - 2;
        int quarter = warp % 4, half = e / 4;
        int buf = 0;
        uint32_t buf_ph[2] = {0, 0};
        bool ok = true;
        int ngroups = (nchunk + ZT_GROUP - 1) / ZT_GROUP;
        for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            ZTile tl = p.tiles[t];
            float hi[CW], lo[CW];
#pragma unroll
            for (int j = 0; j < CW; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
            for (int g = 0; g < ngroups; ++g) {
                if (!mbar_wait(&tfull_bar[buf], buf_ph[buf], &abort_flag, p.err, kDevTimeoutEpi)) { ok = false; break; }
                tc_fence_after();
                uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + buf * (NPL * NB) + half * CW;
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += 8) {
                    uint32_t x[8], y[8];
                    float cc[8];
                    tmem_ld8(tb + 3 * NB + c0, x);
                    tmem_ld8(tb + 2 * NB + c0, y);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; ++j) cc[j] = fmaf(__uint_as_float(x[j]), 0x1p-8f, __uint_as_float(y[j]));
                    tmem_ld8(tb + 1 * NB + c0, x);
                    tmem_ld8(tb + 0 * NB + c0, y);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float c1 = fmaf(cc[j], 0x1p-8f, __uint_as_float(x[j]));
                        float a0 = __uint_as_float(y[j]);
                        float s2 = hi[c0 + j] + a0;
                        float bb = s2 - hi[c0 + j];
                        float er = (hi[c0 + j] - (s2 - bb)) + (a0 - bb);
                        hi[c0 + j] = s2;
                        lo[c0 + j] += er + c1 * 0x1p-8f;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty_bar[buf]);
                buf_ph[buf] ^= 1;
                buf ^= 1;
            }
            if (!ok) break;
            int row = tl.mrow + quarter * 32 + lane;
            bool im = row >= p.Rpad;
            int r = im ? row - p.Rpad : row;
            if (r < p.R) {
                int kp = p.rowk[r], m = p.rowm[r];
                ZPairInfo pi = p.pinfo[(size_t)tl.k * p.nk + kp];
                if (pi.pair >= 0) {
                    const PairDesc pr = p.pairs[pi.pair];
                    int Gx = p.wxyz[3 * tl.w] + pi.g0x - p.ax0, Gy = p.wxyz[3 * tl.w + 1] + pi.g0y - p.ay0,
                        Gz = p.wxyz[3 * tl.w + 2] + pi.g0z - p.az0;
                    int g = -1;
                    if (Gx >= 0 && Gx < p.ad0 && Gy >= 0 && Gy < p.ad1 && Gz >= 0 && Gz < p.ad2)
                        g = p.gtab[(((size_t)pr.qslot * p.ad0 + Gx) * p.ad1 + Gy) * p.ad2 + Gz];
                    if (g >= 0) {
                        int ea = p.aexp[row] - 16;
#pragma unroll
                        for (int j = 0; j < CW; ++j) {
                            int n = tl.nblk * NB + half * CW + j;
                            if (n < pr.nb) {
                                double v = ldexp((double)hi[j] + (double)lo[j], ea + p.eT[(size_t)tl.k * p.nbmax + n]) * p.rs;
                                long long col = pr.col0 + (long long)m * pr.nb + n;
                                double *dst = reinterpret_cast<double *>(p.Z + col * p.RSc + p.nmt + g);
                                dst[im ? 1 : 0] = v;
                            }
                        }
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

}  // namespace

// Host side: geometry, slices, shift lists, tiles and launch for one batch.
int zipw_tc_prepare_and_launch(hfx_ctx *ctx, const ZipwTcInput &in) {
    cudaStream_t st = ctx->stream;
    int rc;
    const int nk = ctx->nk;
    // ---- G1 box and lines over every k' plane-wave list
    int gmin[3] = {1 << 29, 1 << 29, 1 << 29}, gmax[3] = {-(1 << 29), -(1 << 29), -(1 << 29)};
    for (auto &k : ctx->kp)
        for (size_t i = 0; i < k.G.size(); ++i) {
            int x = i % 3;
            gmin[x] = std::min(gmin[x], k.G[i]);
            gmax[x] = std::max(gmax[x], k.G[i]);
        }
    int Bx = gmax[0] - gmin[0] + 1, By = gmax[1] - gmin[1] + 1, Bz = gmax[2] - gmin[2] + 1;
    if (Bz > 16) return set_err(ctx, HFX_EUNSUPPORTED, "plane-wave sphere wider than 16 along b_3");
    std::vector<int> line_of((size_t)Bx * By, -1), lx, ly;
    for (auto &k : ctx->kp)
        for (size_t i = 0; i < k.G.size(); i += 3) line_of[(size_t)(k.G[i] - gmin[0]) * By + (k.G[i + 1] - gmin[1])] = 0;
    for (int x = 0; x < Bx; ++x)
        for (int y = 0; y < By; ++y)
            if (line_of[(size_t)x * By + y] == 0) {
                line_of[(size_t)x * By + y] = (int)lx.size();
                lx.push_back(gmin[0] + x);
                ly.push_back(gmin[1] + y);
            }
    int nL = (int)lx.size(), nLp = (nL + 3) / 4 * 4;
    while ((int)lx.size() < nLp) { lx.push_back(lx[0]); ly.push_back(ly[0]); }
    int KH = nLp * 16, H = nLp / 4;
    // ---- rows (k', m) of every k' that some pair of the batch uses
    std::vector<int> rowk, rowm, rowbase(nk, -1);
    for (int kp = 0; kp < nk; ++kp) {
        rowbase[kp] = (int)rowk.size();
        for (int m = 0; m < ctx->kp[kp].no; ++m) { rowk.push_back(kp); rowm.push_back(m); }
    }
    int R = (int)rowk.size();
    if (R == 0) return HFX_OK;
    int Rpad = (R + 127) / 128 * 128;
    int NBt = std::min(64, (in.nb_max + 15) / 16 * 16);
    int nblk = (in.nb_max + NBt - 1) / NBt;
    // ---- aux lookup tables over the batch's q
    int amin[3] = {1 << 29, 1 << 29, 1 << 29}, amax[3] = {-(1 << 29), -(1 << 29), -(1 << 29)};
    for (int iq : in.qs)
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
    int nq = (int)in.qs.size();
    std::vector<int> gtab((size_t)nq * ad[0] * ad[1] * ad[2], -1);
    for (int s = 0; s < nq; ++s) {
        const std::vector<int> &G = ctx->qp[in.qs[s]].G;
        for (size_t g = 0; g < G.size() / 3; ++g)
            gtab[(((size_t)s * ad[0] + (G[3 * g] - amin[0])) * ad[1] + (G[3 * g + 1] - amin[1])) * ad[2] + (G[3 * g + 2] - amin[2])] = (int)g;
    }
    // ---- pair info (k, k') and the shift lists / tiles per k
    std::vector<ZPairInfo> pinfo((size_t)nk * nk, ZPairInfo{-1, 0, 0, 0});
    for (int i = 0; i < (int)in.pairs.size(); ++i) {
        const PairDesc &pr = in.pairs[i];
        pinfo[(size_t)pr.ik * nk + pr.ikp] = ZPairInfo{i, pr.g0[0], pr.g0[1], pr.g0[2]};
    }
    // W = G - G0 lies in [amin, amax + 1]
    int wd[3] = {ad[0] + 1, ad[1] + 1, ad[2] + 1};
    size_t wvol = (size_t)wd[0] * wd[1] * wd[2];
    int nmt_tiles = 2 * Rpad / ZT_BM;
    std::vector<int> wxyz;
    std::vector<ZTile> tiles;
    std::vector<unsigned char> need;
    std::vector<int> kslot(nk, -1);
    int nslot = 0;
    for (int ik : in.kset) {
        kslot[ik] = nslot++;
        need.assign(wvol * nmt_tiles, 0);
        for (int i = 0; i < (int)in.pairs.size(); ++i) {
            const PairDesc &pr = in.pairs[i];
            if (pr.ik != ik || pr.no == 0) continue;
            const std::vector<int> &G = ctx->qp[pr.iq].G;
            int r0 = rowbase[pr.ikp], r1 = r0 + pr.no;
            int t0 = r0 / ZT_BM, t1 = (r1 - 1) / ZT_BM;
            for (size_t g = 0; g < G.size() / 3; ++g) {
                int w0 = G[3 * g] - pr.g0[0] - amin[0], w1 = G[3 * g + 1] - pr.g0[1] - amin[1], w2 = G[3 * g + 2] - pr.g0[2] - amin[2];
                size_t wi = ((size_t)w0 * wd[1] + w1) * wd[2] + w2;
                for (int t = t0; t <= t1; ++t) {
                    need[wi * nmt_tiles + t] = 1;                    // real rows
                    need[wi * nmt_tiles + t + Rpad / ZT_BM] = 1;     // imaginary rows
                }
            }
        }
        for (size_t wi = 0; wi < wvol; ++wi) {
            bool any = false;
            for (int t = 0; t < nmt_tiles; ++t) any |= need[wi * nmt_tiles + t] != 0;
            if (!any) continue;
            int widx = (int)(wxyz.size() / 3);
            int w2 = (int)(wi % wd[2]), w1 = (int)((wi / wd[2]) % wd[1]), w0 = (int)(wi / ((size_t)wd[1] * wd[2]));
            wxyz.push_back(w0 + amin[0]);
            wxyz.push_back(w1 + amin[1]);
            wxyz.push_back(w2 + amin[2]);
            for (int t = 0; t < nmt_tiles; ++t)
                if (need[wi * nmt_tiles + t])
                    for (int b = 0; b < nblk; ++b) tiles.push_back(ZTile{ik, widx, t * ZT_BM, b});
        }
    }
    if (tiles.empty()) return HFX_OK;
    // ---- device buffers (scratch s_zipw)
    const int Zp = (in.tdim[2] + 7) / 8 * 8;
    size_t bandsz = (size_t)in.tdim[0] * in.tdim[1] * Zp;
    size_t tp_elems = (size_t)nslot * 8 * NPL * 2 * in.nb_max * bandsz;
    size_t a_elems = (size_t)NPL * 2 * Rpad * 2 * KH;
    size_t off = 0;
    auto place = [&](size_t bytes) { size_t o = off; off = (off + bytes + 255) / 256 * 256; return o; };
    size_t o_tp = place(tp_elems * 2), o_a = place(a_elems * 2), o_aexp = place((size_t)2 * Rpad * 4),
           o_eT = place((size_t)nk * in.nb_max * 4), o_rowk = place((size_t)R * 4), o_rowm = place((size_t)R * 4),
           o_line = place((size_t)Bx * By * 4), o_lx = place((size_t)nLp * 4), o_ly = place((size_t)nLp * 4),
           o_gtab = place(gtab.size() * 4), o_pinfo = place(pinfo.size() * sizeof(ZPairInfo)),
           o_w = place(wxyz.size() * 4), o_tiles = place(tiles.size() * sizeof(ZTile)), o_kslot = place((size_t)nk * 4);
    if ((rc = scratch_reserve(ctx, ctx->s_zipw, off))) return rc;
    char *b = reinterpret_cast<char *>(ctx->s_zipw.p);
    auto up = [&](size_t o, const void *src, size_t bytes) {
        return cuda_check(ctx, cudaMemcpyAsync(b + o, src, bytes, cudaMemcpyHostToDevice, st), "zipw tables");
    };
    if ((rc = up(o_rowk, rowk.data(), R * 4)) || (rc = up(o_rowm, rowm.data(), R * 4)) ||
        (rc = up(o_line, line_of.data(), line_of.size() * 4)) || (rc = up(o_lx, lx.data(), nLp * 4)) ||
        (rc = up(o_ly, ly.data(), nLp * 4)) || (rc = up(o_gtab, gtab.data(), gtab.size() * 4)) ||
        (rc = up(o_pinfo, pinfo.data(), pinfo.size() * sizeof(ZPairInfo))) || (rc = up(o_w, wxyz.data(), wxyz.size() * 4)) ||
        (rc = up(o_tiles, tiles.data(), tiles.size() * sizeof(ZTile))) || (rc = up(o_kslot, kslot.data(), nk * 4)))
        return rc;
    __nv_bfloat16 *Tp = reinterpret_cast<__nv_bfloat16 *>(b + o_tp), *A = reinterpret_cast<__nv_bfloat16 *>(b + o_a);
    int *aexp = reinterpret_cast<int *>(b + o_aexp), *eT = reinterpret_cast<int *>(b + o_eT);
    cudaMemsetAsync(aexp, 0, (size_t)2 * Rpad * 4, st);
    cudaMemsetAsync(A, 0, a_elems * 2, st);
    c_slices_kernel<<<R, 256, 0, st>>>(in.d_ck, in.d_Gk, in.d_npw, reinterpret_cast<int *>(b + o_rowk),
                                       reinterpret_cast<int *>(b + o_rowm), reinterpret_cast<int *>(b + o_line), gmin[0], gmin[1],
                                       gmin[2], By, KH, Rpad, A, aexp);
    t_slices_kernel<<<dim3(in.nb_max, nk), 256, 0, st>>>(in.d_Tk, in.d_nb, in.tdim[0], in.tdim[1], in.tdim[2], Zp, in.nb_max,
                                                         reinterpret_cast<int *>(b + o_kslot), Tp, eT);
    if ((rc = cuda_check(ctx, cudaGetLastError(), "zipw slices"))) return rc;
    // ---- tensor maps
    CUtensorMap mA, mT;
    if ((rc = make_map_2d(ctx, &mA, A, (long long)NPL * 2 * Rpad, 2LL * KH, ZT_BM))) return rc;
    unsigned long long dims[5] = {(unsigned long long)Zp, (unsigned long long)in.tdim[1], (unsigned long long)in.tdim[0],
                                  (unsigned long long)in.nb_max, (unsigned long long)nslot * 8 * NPL * 2};
    unsigned long long strides[4] = {(unsigned long long)Zp * 2, (unsigned long long)Zp * in.tdim[1] * 2,
                                     (unsigned long long)bandsz * 2, (unsigned long long)bandsz * in.nb_max * 2};
    unsigned int box[5] = {16, 1, 1, (unsigned int)NBt, 1};
    if ((rc = make_map_5d(ctx, &mT, Tp, dims, strides, box, 32))) return rc;
    ZParams p;
    p.tiles = reinterpret_cast<ZTile *>(b + o_tiles);
    p.ntiles = (int)tiles.size();
    p.wxyz = reinterpret_cast<int *>(b + o_w);
    p.pinfo = reinterpret_cast<ZPairInfo *>(b + o_pinfo);
    p.pairs = in.d_pairs;
    p.gtab = reinterpret_cast<int *>(b + o_gtab);
    p.ax0 = amin[0]; p.ay0 = amin[1]; p.az0 = amin[2];
    p.ad0 = ad[0]; p.ad1 = ad[1]; p.ad2 = ad[2];
    p.rowk = reinterpret_cast<int *>(b + o_rowk);
    p.rowm = reinterpret_cast<int *>(b + o_rowm);
    p.aexp = aexp;
    p.eT = eT;
    p.kslot = reinterpret_cast<int *>(b + o_kslot);
    p.line_x = reinterpret_cast<int *>(b + o_lx);
    p.line_y = reinterpret_cast<int *>(b + o_ly);
    p.Z = in.d_Z;
    p.RSc = in.RSc;
    p.nmt = ctx->nmt;
    p.nk = nk;
    p.R = R;
    p.Rpad = Rpad;
    p.H = H;
    p.KH = KH;
    p.nbmax = in.nb_max;
    p.gz0 = gmin[2];
    p.tlo0 = in.tlo[0]; p.tlo1 = in.tlo[1]; p.tlo2 = in.tlo[2];
    p.rs = 1.0 / sqrt(ctx->omega);
    p.err = ctx->d_err;
    int grid = std::min<int>(num_sms(), p.ntiles);
    auto go = [&](auto kern, int nb) {
        size_t smem = (size_t)ZT_STAGES * NPL * (ZT_A_PLANE + 4 * nb * 32) + 1024;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (in.ev_gemm0) cudaEventRecord(in.ev_gemm0, st);
        kern<<<grid, 64 + 32 * ZT_EPI, smem, st>>>(mA, mT, p);
        if (in.ev_gemm1) cudaEventRecord(in.ev_gemm1, st);
    };
    switch (NBt) {
    case 16: go(zipw_tc_kernel<16>, 16); break;
    case 32: go(zipw_tc_kernel<32>, 32); break;
    case 48: go(zipw_tc_kernel<48>, 48); break;
    default: go(zipw_tc_kernel<64>, 64); break;
    }
    return cuda_check(ctx, cudaGetLastError(), "zipw tensor-core kernel");
}

}  // namespace hfx
