// k_cgemm_tc.cu -- complex products on the tensor cores in exact slice
// arithmetic, for the two dense products of stage 1:
//
//   T_n(K)      = sum_{G2} Theta_{K - G2} c_{G2}(n)                      (Sec. III.B)
//   Z^MT_I(m,n) = e^{-i q.tau_a} sum_{lm p} conj(A_{lmp}(m, k')) B_k[I, lmp, n]   (Sec. III.A)
//
// with B_k[I, lmp, n] = sum_{l'm'p'} G(LM; lm; l'm') R_{a L p; lp, l'p'} A_{l'm'p'}(n, k)
// (transformed by the multipole transform where the block-sparse form is used).
//
// General form: out[rowoff(r) + coloff(g, c)] = phase(g, c) * sum_K A[r, K] B_c[K].
// A rows hold [Re | Im] of one complex row over the reduction index; every
// complex output column is a pair of B rows (Re row, Im row) that carries the
// real embedding of the second factor.  Operands are four-slice fixed-point
// BF16 planes with per-row exponents (tc_ptx.cuh); the ten slice products are
// summed exactly per weight class on the tensor cores (K groups of 256) and
// combined on the CUDA cores into a compensated FP32 pair.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "tc_ptx.cuh"

namespace hfx {

using namespace tc;

namespace {

constexpr int CG_BM = 128, CG_BN = 64, CG_KC = 64;
constexpr int CG_A_PLANE = CG_BM * CG_KC * 2;              // 16 KB
constexpr int CG_B_PLANE = CG_BN * CG_KC * 2;              // 8 KB
constexpr int CG_STAGE = NPL * (CG_A_PLANE + CG_B_PLANE);   // 96 KB
constexpr int CG_STAGES = 2;
constexpr int CG_GROUP = 4;                                // 64-K chunks per exact group (256)
constexpr int CG_TMEM = 512;                               // 2 buffers x 4 classes x 64 columns
constexpr int CG_EPI = 8;

struct CgTile { int arow, brow, grp, phb, nchunk, pad; };

struct CgParams {
    const CgTile *tiles;
    int ntiles;
    const int *aexp, *bexp;          // per A row, per B row
    const long long *rowoff;         // per A row (double2 units); < 0: no output
    const long long *coloff;         // [grp * col_gstride + pair] (double2 units); < 0: no output
    long long col_gstride;
    const float4 *phase;             // optional: phase[phb + pkey[pair]], split (hi re, lo re, hi im, lo im)
    const int *pkey;
    double2 *out;
    long long RA, RB;                // rows per slice plane of A and B
    int *err;
};

// warp 0: TMA producer; warp 1: MMA issuer; warps 2..9: epilogue
// (TMEM lane quarter = warp % 4, column half = (warp - 2) / 4)
__global__ void __launch_bounds__(64 + 32 * CG_EPI, 1) cgemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                    const __grid_constant__ CUtensorMap tmB,
                                                                    CgParams p) {
    extern __shared__ __align__(1024) unsigned char cg_smem[];
    uintptr_t base = (reinterpret_cast<uintptr_t>(cg_smem) + 1023) & ~(uintptr_t)1023;
    unsigned char *stages = reinterpret_cast<unsigned char *>(base);
    __shared__ uint64_t full_bar[CG_STAGES], empty_bar[CG_STAGES], tfull_bar[2], tempty_bar[2], mma_done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < CG_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], CG_EPI);
        }
        mbar_init(&mma_done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_slot, CG_TMEM);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            for (int t = blockIdx.x; t < p.ntiles && !abort_flag; t += gridDim.x) {
                const CgTile tl = p.tiles[t];
                bool stop = false;
                for (int kc = 0; kc < tl.nchunk; ++kc) {
                    if (!mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, p.err, kDevTimeoutTma)) { stop = true; break; }
                    unsigned char *st = stages + (size_t)s * CG_STAGE;
                    mbar_expect_tx(&full_bar[s], CG_STAGE);
#pragma unroll
                    for (int pl = 0; pl < NPL; ++pl) {
                        tma_load_2d(saddr(st + pl * CG_A_PLANE), &tmA, &full_bar[s], kc * CG_KC, (int)(pl * p.RA + tl.arow));
                        tma_load_2d(saddr(st + NPL * CG_A_PLANE + pl * CG_B_PLANE), &tmB, &full_bar[s], kc * CG_KC,
                                    (int)(pl * p.RB + tl.brow));
                    }
                    ++issued;
                    if (++s == CG_STAGES) { s = 0; ph ^= 1; }
                }
                if (stop) break;
            }
            if (abort_flag) {
                for (int i = 0; i < CG_STAGES && i < issued; ++i) mbar_drain(&full_bar[i], 0), mbar_drain(&full_bar[i], 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int buf = 0;
            uint32_t buf_ph[2] = {0, 0};
            // A slice a times the B slices b = 0 .. 3 - a stacked in N (the B planes
            // are contiguous) lands in the class columns (a + b) CG_BN: four MMAs
            // per K step cover the ten slice products
            constexpr uint32_t id1 = idesc_bf16(CG_BM, CG_BN), id2 = idesc_bf16(CG_BM, 2 * CG_BN);
            constexpr uint32_t id3 = idesc_bf16(CG_BM, 3 * CG_BN), id4 = idesc_bf16(CG_BM, 4 * CG_BN);
            bool ok = true;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
                const int nchunk = p.tiles[t].nchunk;
                for (int g0 = 0; g0 < nchunk && ok; g0 += CG_GROUP) {
                    if (!mbar_wait(&tempty_bar[buf], buf_ph[buf] ^ 1, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                    tc_fence_after();
                    uint32_t dt = tmem + buf * (NPL * CG_BN);
                    for (int kc = g0; kc < min(nchunk, g0 + CG_GROUP); ++kc) {
                        if (!mbar_wait(&full_bar[s], ph, &abort_flag, p.err, kDevTimeoutMma)) { ok = false; break; }
                        tc_fence_after();
                        unsigned char *st = stages + (size_t)s * CG_STAGE;
                        uint32_t a0 = saddr(st), b0 = saddr(st + NPL * CG_A_PLANE);
                        const bool first = kc == g0;
#pragma unroll
                        for (int ks = 0; ks < CG_KC / 16; ++ks) {
                            const uint64_t e0 = desc_sw128(b0) + 2 * ks;
                            // the a = 0 MMA of a group's first K step overwrites every class
                            umma_bf16(dt, desc_sw128(a0) + 2 * ks, e0, id4, (first && ks == 0) ? 0u : 1u);
                            umma_bf16(dt + CG_BN, desc_sw128(a0 + CG_A_PLANE) + 2 * ks, e0, id3, 1u);
                            umma_bf16(dt + 2 * CG_BN, desc_sw128(a0 + 2 * CG_A_PLANE) + 2 * ks, e0, id2, 1u);
                            umma_bf16(dt + 3 * CG_BN, desc_sw128(a0 + 3 * CG_A_PLANE) + 2 * ks, e0, id1, 1u);
                        }
                        umma_commit(&empty_bar[s]);
                        if (++s == CG_STAGES) { s = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    umma_commit(&tfull_bar[buf]);
                    buf_ph[buf] ^= 1;
                    buf ^= 1;
                }
            }
            umma_drain(&mma_done);
        }
    } else {
        int e = warp - 2;
        int quarter = warp % 4, half = e / 4;
        int buf = 0;
        uint32_t buf_ph[2] = {0, 0};
        bool ok = true;
        for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            const CgTile tl = p.tiles[t];
            int ngroups = (tl.nchunk + CG_GROUP - 1) / CG_GROUP;
            // the output's row offset and row exponent, and per column pair l of
            // this half (held by lane l < 16, shuffled in the store loop) its
            // offset, the two column exponents and the phase: fetched now so that
            // the loads overlap the K loop
            const int r = tl.arow + quarter * 32 + lane;
            const long long ro = p.rowoff[r];
            const int ea = ro >= 0 ? p.aexp[r] - 16 : 0;
            long long co_l = -1;
            int br_l = 0, bi_l = 0;
            float4 f_l = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
            if (lane < 16) {
                const int c = tl.brow + half * 32 + 2 * lane;
                co_l = p.coloff[(long long)tl.grp * p.col_gstride + (c >> 1)];
                br_l = p.bexp[c];
                bi_l = p.bexp[c + 1];
                if (p.phase) f_l = p.phase[tl.phb + p.pkey[c >> 1]];
            }
            uint64_t hi[16], lo[16];   // packed pairs of columns
#pragma unroll
            for (int j = 0; j < 16; ++j) { hi[j] = 0; lo[j] = 0; }
            for (int g = 0; g < ngroups; ++g) {
                if (!mbar_wait(&tfull_bar[buf], buf_ph[buf], &abort_flag, p.err, kDevTimeoutEpi)) { ok = false; break; }
                tc_fence_after();
                uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + buf * (NPL * CG_BN) + half * 32;
#pragma unroll
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    uint32_t a0[16], a1[16], a2[16], a3[16];
                    tmem_ld16(tb + 0 * CG_BN + c0, a0);
                    tmem_ld16(tb + 1 * CG_BN + c0, a1);
                    tmem_ld16(tb + 2 * CG_BN + c0, a2);
                    tmem_ld16(tb + 3 * CG_BN + c0, a3);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; j += 2)
                        class_accumulate2(f2_pack(a0[j], a0[j + 1]), f2_pack(a1[j], a1[j + 1]), f2_pack(a2[j], a2[j + 1]),
                                          f2_pack(a3[j], a3[j + 1]), hi[(c0 + j) / 2], lo[(c0 + j) / 2]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty_bar[buf]);
                buf_ph[buf] ^= 1;
                buf ^= 1;
            }
            if (!ok) break;
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
                const int src = j / 2;
                const long long co = __shfl_sync(0xffffffffu, co_l, src);
                const int br = __shfl_sync(0xffffffffu, br_l, src), bi = __shfl_sync(0xffffffffu, bi_l, src);
                const float2 h = f2_unpack(hi[j / 2]), l = f2_unpack(lo[j / 2]);
                double re, im;
                if (p.phase) {
                    // (re + i im) e^{-i q.tau} in double-FP32 on the FP32 units (about
                    // 2^-44 relative; the projections are sliced to 2^-32 next), both
                    // parts first brought to the larger of their two column scales
                    float4 f;
                    f.x = __shfl_sync(0xffffffffu, f_l.x, src);
                    f.y = __shfl_sync(0xffffffffu, f_l.y, src);
                    f.z = __shfl_sync(0xffffffffu, f_l.z, src);
                    f.w = __shfl_sync(0xffffffffu, f_l.w, src);
                    const int sm = max(br, bi);
                    const float sr = pow2f_neg(br - sm), si = pow2f_neg(bi - sm);
                    float rh, rl, ih, il;
                    two_sum(h.x * sr, l.x * sr, rh, rl);
                    two_sum(h.y * si, l.y * si, ih, il);
                    float Sr = 0.0f, Er = 0.0f, Si = 0.0f, Ei = 0.0f;
                    df_mac(rh, rl, f.x, f.y, Sr, Er);
                    df_mac(-ih, -il, f.z, f.w, Sr, Er);
                    df_mac(rh, rl, f.z, f.w, Si, Ei);
                    df_mac(ih, il, f.x, f.y, Si, Ei);
                    re = f32pair_to_f64(Sr, Er, ea + sm);
                    im = f32pair_to_f64(Si, Ei, ea + sm);
                } else {
                    re = f32pair_to_f64(h.x, l.x, ea + br);
                    im = f32pair_to_f64(h.y, l.y, ea + bi);
                }
                if (ro >= 0 && co >= 0) __stcs(p.out + ro + co, make_double2(re, im));   // streaming: keep the operands in L2
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, CG_TMEM);
    }
}

// ------------------------------------------------------------- operand slices
__device__ __forceinline__ void put_row(__nv_bfloat16 *X, long long plane, long long row, int W, int col, double v, int e) {
    __nv_bfloat16 s[NPL];
    slice4(v, e, s);
#pragma unroll
    for (int pl = 0; pl < NPL; ++pl) X[pl * plane + row * W + col] = s[pl];
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long m) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}

// A rows of the step-function product: row p = point K of the T box,
// [Re | Im] Theta_{K - U_g} over the common plane-wave list U.
__global__ void theta_toep_kernel(const double2 *__restrict__ theta, int dlo0, int dlo1, int dlo2, int dd1, int dd2,
                                  int tlo0, int tlo1, int tlo2, int td0, int td1, int td2, const int *__restrict__ uoff,
                                  int NU, int Kh, long long RA, __nv_bfloat16 *__restrict__ A, int *__restrict__ aexp) {
    long long p = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x % 32;
    if (p >= RA) return;
    const int W = 2 * Kh;
    const long long plane = RA * W;
    long long box = (long long)td0 * td1 * td2;
    long long dbase = -1;
    if (p < box) {
        int kz = (int)(p % td2), ky = (int)((p / td2) % td1), kx = (int)(p / ((long long)td1 * td2));
        dbase = ((long long)(tlo0 + kx - dlo0) * dd1 + (tlo1 + ky - dlo1)) * dd2 + (tlo2 + kz - dlo2);
    }
    unsigned long long mx = 0;
    if (dbase >= 0)
        for (int g = lane; g < NU; g += 32) {
            double2 t = theta[dbase - uoff[g]];
            mx = max(mx, max(abs_bits(t.x), abs_bits(t.y)));
        }
    int e = line_exp_bits(warp_max(mx));
    if (lane == 0) aexp[p] = e;
    for (int g = lane; g < Kh; g += 32) {
        double2 t = (dbase >= 0 && g < NU) ? theta[dbase - uoff[g]] : make_double2(0.0, 0.0);
        put_row(A, plane, p, W, g, t.x, e);
        put_row(A, plane, p, W, Kh + g, t.y, e);
    }
}

// B row pair t = (k, n) of the step-function product: Re row [c_r | -c_i],
// Im row [c_i | c_r] on the common list U (buffer zeroed beforehand).
__global__ void cband_slices_kernel(const double2 *const *__restrict__ ck, const int *__restrict__ npw_k,
                                    const int *__restrict__ uidx, const long long *__restrict__ uidx_off,
                                    const int *__restrict__ rk, const int *__restrict__ rn, int npairs, int Kh,
                                    long long RB, __nv_bfloat16 *__restrict__ B, int *__restrict__ bexp) {
    int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x % 32;
    if (t >= npairs) return;
    const int k = rk[t], n = rn[t], npw = npw_k[k];
    const double2 *c = ck[k] + (size_t)n * npw;
    const int *ui = uidx + uidx_off[k];
    const int W = 2 * Kh;
    const long long plane = RB * W;
    unsigned long long mx = 0;
    for (int i = lane; i < npw; i += 32) mx = max(mx, max(abs_bits(c[i].x), abs_bits(c[i].y)));
    int e = line_exp_bits(warp_max(mx));
    if (lane == 0) { bexp[2 * t] = e; bexp[2 * t + 1] = e; }
    for (int i = lane; i < npw; i += 32) {
        int u = ui[i];
        double cr = c[i].x, ci = c[i].y;
        put_row(B, plane, 2 * t, W, u, cr, e);
        put_row(B, plane, 2 * t, W, Kh + u, -ci, e);
        put_row(B, plane, 2 * t + 1, W, u, ci, e);
        put_row(B, plane, 2 * t + 1, W, Kh + u, cr, e);
    }
}

// A rows of the muffin-tin product, block b = (k, a): row n * nLMP + (LM P + i),
// [Re | Im] B_k[(a LM i), lmp, n] over lmp.
__global__ void bk_slices_kernel(const double2 *const *__restrict__ Bk, const int *__restrict__ blk_k,
                                 const int *__restrict__ blk_a, const long long *__restrict__ blk_row0,
                                 const int *__restrict__ nb_k, int nLMP, int nlmp, int Kh, long long RA,
                                 __nv_bfloat16 *__restrict__ A, int *__restrict__ aexp) {
    const int b = blockIdx.y, k = blk_k[b], a = blk_a[b], nb = nb_k[k];
    const int rows = nb * nLMP, rows_pad = (rows + CG_BM - 1) / CG_BM * CG_BM;
    const int W = 2 * Kh;
    const long long plane = RA * W;
    int lane = threadIdx.x % 32, wpb = blockDim.x / 32;
    for (int ir = blockIdx.x * wpb + threadIdx.x / 32; ir < rows_pad; ir += gridDim.x * wpb) {
        long long r = blk_row0[b] + ir;
        const double2 *src = nullptr;
        if (ir < rows) {
            int n = ir / nLMP, lmi = ir % nLMP;
            src = Bk[k] + ((size_t)(a * nLMP + lmi) * nlmp) * nb + n;
        }
        unsigned long long mx = 0;
        if (src)
            for (int g = lane; g < nlmp; g += 32) mx = max(mx, max(abs_bits(src[(size_t)g * nb].x), abs_bits(src[(size_t)g * nb].y)));
        int e = line_exp_bits(warp_max(mx));
        if (lane == 0) aexp[r] = e;
        for (int g = lane; g < Kh; g += 32) {
            double2 v = (src && g < nlmp) ? src[(size_t)g * nb] : make_double2(0.0, 0.0);
            put_row(A, plane, r, W, g, v.x, e);
            put_row(A, plane, r, W, Kh + g, v.y, e);
        }
    }
}

// B row pairs of the muffin-tin product, atom block a: pair ip = (k', m),
// Re row [Y_r | Y_i], Im row [-Y_i | Y_r] with Y = A_{lmp}(m, k') of atom a
// (their product with an A row is sum_K X conj(Y)).
__global__ void ak_slices_kernel(const double2 *const *__restrict__ Ak, const int *__restrict__ pk,
                                 const int *__restrict__ pm, int npairs_a, int npairs_pad, const long long *__restrict__ brow0,
                                 int n_atoms, int nlmp, int Kh, long long RB, __nv_bfloat16 *__restrict__ B,
                                 int *__restrict__ bexp) {
    const int a = blockIdx.y;
    const int W = 2 * Kh;
    const long long plane = RB * W;
    int lane = threadIdx.x % 32, wpb = blockDim.x / 32;
    for (int ip = blockIdx.x * wpb + threadIdx.x / 32; ip < npairs_pad; ip += gridDim.x * wpb) {
        long long r = brow0[a] + 2LL * ip;
        const double2 *y = nullptr;
        if (ip < npairs_a) y = Ak[pk[ip]] + ((size_t)pm[ip] * n_atoms + a) * nlmp;
        unsigned long long mx = 0;
        if (y)
            for (int g = lane; g < nlmp; g += 32) mx = max(mx, max(abs_bits(y[g].x), abs_bits(y[g].y)));
        int e = line_exp_bits(warp_max(mx));
        if (lane == 0) { bexp[r] = e; bexp[r + 1] = e; }
        for (int g = lane; g < Kh; g += 32) {
            double2 v = (y && g < nlmp) ? y[g] : make_double2(0.0, 0.0);
            put_row(B, plane, r, W, g, v.x, e);
            put_row(B, plane, r, W, Kh + g, v.y, e);
            put_row(B, plane, r + 1, W, g, -v.y, e);
            put_row(B, plane, r + 1, W, Kh + g, v.x, e);
        }
    }
}

int grid_rows(long long rows, int per_block) {
    long long g = (rows + per_block - 1) / per_block;
    return (int)std::max<long long>(1, std::min<long long>(g, 1 << 20));
}

// Tensor maps, parameters and launch of one product.
int launch_cgemm(hfx_ctx *ctx, const __nv_bfloat16 *A, long long RA, const __nv_bfloat16 *B, long long RB, int Kw,
                 CgParams p) {
    int rc;
    CUtensorMap mA, mB;
    if ((rc = make_map_2d(ctx, &mA, A, (long long)NPL * RA, Kw, CG_BM))) return rc;
    if ((rc = make_map_2d(ctx, &mB, B, (long long)NPL * RB, Kw, CG_BN))) return rc;
    if (p.ntiles == 0) return HFX_OK;
    p.RA = RA;
    p.RB = RB;
    p.err = ctx->d_err;
    size_t smem = (size_t)CG_STAGES * CG_STAGE + 1024;
    cudaFuncSetAttribute(cgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int grid = std::min(num_sms(), p.ntiles);
    cgemm_kernel<<<grid, 64 + 32 * CG_EPI, smem, ctx->stream>>>(mA, mB, p);
    return cuda_check(ctx, cudaGetLastError(), "slice product kernel");
}

}  // namespace

// =====================================================================
// T_n(K) of every k of kset:  T_k[n][K] at d_T + toff[k] + n * box.
// Plan: the common plane-wave list, the operand rows and the tiles (host
// tables, uploaded once with the build plan); run: the operand slices and the
// product, every build.
int thetapsi_tc_plan(hfx_ctx *ctx, const std::vector<int> &kset, const int ddim[3], const int tdim[3],
                     const std::vector<size_t> &toff, HostArena &tab, TpPlan &tp) {
    tp = TpPlan();
    if (kset.empty()) return HFX_OK;
    const long long box = (long long)tdim[0] * tdim[1] * tdim[2];
    // common plane-wave list U over every k of the mesh (not only kset: the
    // operands, and so the rounding, of T_k do not depend on which k are built)
    int gmin[3] = {1 << 29, 1 << 29, 1 << 29}, gmax[3] = {-(1 << 29), -(1 << 29), -(1 << 29)};
    for (int k = 0; k < ctx->nk; ++k)
        for (size_t i = 0; i < ctx->kp[k].G.size(); ++i) {
            int x = i % 3;
            gmin[x] = std::min(gmin[x], ctx->kp[k].G[i]);
            gmax[x] = std::max(gmax[x], ctx->kp[k].G[i]);
        }
    int bd[3];
    for (int x = 0; x < 3; ++x) bd[x] = gmax[x] >= gmin[x] ? gmax[x] - gmin[x] + 1 : 1;
    std::vector<int> dense((size_t)bd[0] * bd[1] * bd[2], -1), uoff, uidx;
    std::vector<long long> uidx_off(ctx->nk, 0);
    for (int k = 0; k < ctx->nk; ++k) {
        const std::vector<int> &G = ctx->kp[k].G;
        uidx_off[k] = (long long)uidx.size();
        for (size_t i = 0; i + 2 < G.size(); i += 3) {
            size_t d = ((size_t)(G[i] - gmin[0]) * bd[1] + (G[i + 1] - gmin[1])) * bd[2] + (G[i + 2] - gmin[2]);
            if (dense[d] < 0) {
                dense[d] = (int)uoff.size();
                uoff.push_back((G[i] * ddim[1] + G[i + 1]) * ddim[2] + G[i + 2]);
            }
            uidx.push_back(dense[d]);
        }
    }
    const int NU = (int)uoff.size();
    if (NU == 0) return HFX_OK;
    const int Kh = (NU + 63) / 64 * 64, Kw = 2 * Kh;
    const long long RA = (box + CG_BM - 1) / CG_BM * CG_BM;
    std::vector<int> rk, rn;
    std::vector<long long> coloff;
    for (int k : kset)
        for (int n = 0; n < ctx->kp[k].nb; ++n) {
            rk.push_back(k);
            rn.push_back(n);
            coloff.push_back((long long)toff[k] + (long long)n * box);
        }
    const int npairs = (int)rk.size();
    const long long RB = (2LL * npairs + CG_BN - 1) / CG_BN * CG_BN;
    while ((long long)coloff.size() < RB / 2) coloff.push_back(-1);
    std::vector<long long> rowoff(RA);
    for (long long p = 0; p < RA; ++p) rowoff[p] = p < box ? p : -1;
    std::vector<CgTile> tiles;
    for (long long a = 0; a < RA; a += CG_BM)
        for (long long b = 0; b < RB; b += CG_BN) tiles.push_back(CgTile{(int)a, (int)b, 0, 0, Kw / CG_KC, 0});
    std::vector<const double2 *> hc(ctx->nk, nullptr);
    std::vector<int> hnpw(ctx->nk, 0);
    for (int k = 0; k < ctx->nk; ++k) { hc[k] = ctx->kp[k].d_c; hnpw[k] = ctx->kp[k].npw; }
    tp.o_uo = tab.put(uoff);
    tp.o_ui = tab.put(uidx);
    tp.o_uio = tab.put(uidx_off);
    tp.o_rk = tab.put(rk);
    tp.o_rn = tab.put(rn);
    tp.o_co = tab.put(coloff);
    tp.o_ro = tab.put(rowoff);
    tp.o_ti = tab.put(tiles);
    tp.o_hc = tab.put(hc);
    tp.o_np = tab.put(hnpw);
    Layout lay;
    tp.s_A = lay.place((size_t)NPL * RA * Kw * 2);
    tp.s_B = lay.place((size_t)NPL * RB * Kw * 2);
    tp.s_ae = lay.place(RA * 4);
    tp.s_be = lay.place(RB * 4);
    tp.scratch_bytes = lay.off;
    tp.NU = NU;
    tp.Kh = Kh;
    tp.RA = RA;
    tp.RB = RB;
    tp.npairs = npairs;
    tp.ntiles = (int)tiles.size();
    tp.ok = true;
    return HFX_OK;
}

int thetapsi_tc_run(hfx_ctx *ctx, const TpPlan &tp, const char *dtab, char *dscr, const double2 *d_theta, const int dlo[3],
                    const int ddim[3], const int tlo[3], const int tdim[3], double2 *d_T, int *nlaunch) {
    if (!tp.ok) return HFX_OK;
    int rc;
    const int Kw = 2 * tp.Kh;
    __nv_bfloat16 *A = reinterpret_cast<__nv_bfloat16 *>(dscr + tp.s_A), *B = reinterpret_cast<__nv_bfloat16 *>(dscr + tp.s_B);
    int *ae = reinterpret_cast<int *>(dscr + tp.s_ae), *be = reinterpret_cast<int *>(dscr + tp.s_be);
    cudaMemsetAsync(B, 0, (size_t)NPL * tp.RB * Kw * 2, ctx->stream);
    cudaMemsetAsync(be, 0, tp.RB * 4, ctx->stream);
    theta_toep_kernel<<<grid_rows(tp.RA, 8), 256, 0, ctx->stream>>>(
        d_theta, dlo[0], dlo[1], dlo[2], ddim[1], ddim[2], tlo[0], tlo[1], tlo[2], tdim[0], tdim[1], tdim[2],
        reinterpret_cast<const int *>(dtab + tp.o_uo), tp.NU, tp.Kh, tp.RA, A, ae);
    cband_slices_kernel<<<grid_rows(tp.npairs, 8), 256, 0, ctx->stream>>>(
        reinterpret_cast<const double2 *const *>(dtab + tp.o_hc), reinterpret_cast<const int *>(dtab + tp.o_np),
        reinterpret_cast<const int *>(dtab + tp.o_ui), reinterpret_cast<const long long *>(dtab + tp.o_uio),
        reinterpret_cast<const int *>(dtab + tp.o_rk), reinterpret_cast<const int *>(dtab + tp.o_rn), tp.npairs, tp.Kh,
        tp.RB, B, be);
    if ((rc = cuda_check(ctx, cudaGetLastError(), "step-function product slices"))) return rc;
    CgParams p{};
    p.tiles = reinterpret_cast<const CgTile *>(dtab + tp.o_ti);
    p.ntiles = tp.ntiles;
    p.aexp = ae;
    p.bexp = be;
    p.rowoff = reinterpret_cast<const long long *>(dtab + tp.o_ro);
    p.coloff = reinterpret_cast<const long long *>(dtab + tp.o_co);
    p.col_gstride = 0;
    p.phase = nullptr;
    p.pkey = nullptr;
    p.out = d_T;
    if (nlaunch) *nlaunch += 3;
    return launch_cgemm(ctx, A, tp.RA, B, tp.RB, Kw, p);
}

// =====================================================================
// Z^MT on the tensor cores.  Plan (per build): rows of the B_k slices (A
// operand, per (k, a) block) and of the A_{k'} slices (B operand, row pairs
// per atom block); run: the slices, every build.  Per batch: output offsets,
// phases and tiles (plan) and the product (run).
int zmt_tc_plan(hfx_ctx *ctx, const std::vector<int> &kset, const std::vector<double2 *> &hB, long long RSc, int N0,
                int sparse, HostArena &tab, ZmtPlan &zs) {
    const int nk = ctx->nk, na = ctx->sys.n_atoms, P = ctx->P, nLM = ctx->nLM, nLMP = nLM * P, nlmp = ctx->nlmp;
    zs = ZmtPlan();
    zs.Kh = (nlmp + 63) / 64 * 64;
    const int Kw = 2 * zs.Kh;
    // A operand blocks (k, a)
    std::vector<int> blk_k, blk_a;
    std::vector<long long> blk_row0;
    zs.blk_row0.assign((size_t)nk * na, -1);
    zs.blk_rows.assign((size_t)nk * na, 0);
    long long RA = 0;
    for (int k : kset)
        for (int a = 0; a < na; ++a) {
            long long rows = (long long)ctx->kp[k].nb * nLMP;
            if (rows == 0) continue;
            blk_k.push_back(k);
            blk_a.push_back(a);
            blk_row0.push_back(RA);
            zs.blk_row0[(size_t)k * na + a] = RA;
            zs.blk_rows[(size_t)k * na + a] = rows;
            RA += (rows + CG_BM - 1) / CG_BM * CG_BM;
        }
    if (RA == 0) return HFX_OK;
    std::vector<long long> rowoff(RA, -1);
    for (size_t b = 0; b < blk_k.size(); ++b) {
        int k = blk_k[b], a = blk_a[b];
        for (int n = 0; n < ctx->kp[k].nb; ++n)
            for (int LM = 0; LM < nLM; ++LM)
                for (int i = 0; i < P; ++i) {
                    int ch = a * nLM + LM;
                    int zrow = sparse ? (i == 0 ? N0 + ch : ch * (P - 1) + i - 1) : ch * P + i;
                    rowoff[blk_row0[b] + (long long)n * nLMP + LM * P + i] = (long long)n * RSc + zrow;
                }
    }
    // B operand: pairs (k', m) in every atom block
    std::vector<int> pk, pm;
    zs.kbase.assign(nk, 0);
    for (int kp = 0; kp < nk; ++kp) {
        zs.kbase[kp] = (int)pk.size();
        for (int m = 0; m < ctx->kp[kp].nom; ++m) { pk.push_back(kp); pm.push_back(m); }
    }
    zs.npairs_a = (int)pk.size();
    if (zs.npairs_a == 0) return HFX_OK;
    zs.npairs_pad = (zs.npairs_a + CG_BN / 2 - 1) / (CG_BN / 2) * (CG_BN / 2);
    const long long RB = (long long)na * 2 * zs.npairs_pad;
    std::vector<long long> brow0(na);
    for (int a = 0; a < na; ++a) brow0[a] = (long long)a * 2 * zs.npairs_pad;
    std::vector<int> pkey(RB / 2);
    for (int a = 0; a < na; ++a)
        for (int ip = 0; ip < zs.npairs_pad; ++ip) pkey[(size_t)a * zs.npairs_pad + ip] = ip < zs.npairs_a ? pk[ip] : 0;
    zs.RA = RA;
    zs.RB = RB;
    zs.blocks.clear();
    for (size_t b = 0; b < blk_k.size(); ++b) zs.blocks.push_back({blk_k[b], blk_a[b]});
    std::vector<const double2 *> hA(nk), hBc(nk);
    std::vector<int> hnb(nk);
    for (int k = 0; k < nk; ++k) { hA[k] = ctx->kp[k].d_Am; hBc[k] = hB[k]; hnb[k] = ctx->kp[k].nb; }
    zs.o_ro = tab.put(rowoff);
    zs.o_pk = tab.put(pkey);
    zs.o_bk = tab.put(blk_k);
    zs.o_ba = tab.put(blk_a);
    zs.o_br = tab.put(blk_row0);
    zs.o_nb = tab.put(hnb);
    zs.o_hb = tab.put(hBc);
    zs.o_ha = tab.put(hA);
    zs.o_pk2 = tab.put(pk);
    zs.o_pm = tab.put(pm);
    zs.o_br0 = tab.put(brow0);
    zs.nblocks = (int)blk_k.size();
    int nbmax = 0;
    for (int k : kset) nbmax = std::max(nbmax, ctx->kp[k].nb);
    zs.maxrows = ((long long)nbmax * nLMP + CG_BM - 1) / CG_BM * CG_BM;
    Layout lay;
    zs.s_A = lay.place((size_t)NPL * RA * Kw * 2);
    zs.s_B = lay.place((size_t)NPL * RB * Kw * 2);
    zs.s_ae = lay.place(RA * 4);
    zs.s_be = lay.place(RB * 4);
    zs.scratch_bytes = lay.off;
    zs.ok = true;
    return HFX_OK;
}

int zmt_tc_run_prepare(hfx_ctx *ctx, const ZmtPlan &zs, const char *dtab, char *dscr, int *nlaunch) {
    if (!zs.ok) return HFX_OK;
    const int na = ctx->sys.n_atoms, nLMP = ctx->nLM * ctx->P, nlmp = ctx->nlmp;
    bk_slices_kernel<<<dim3(grid_rows(zs.maxrows, 8), (unsigned)zs.nblocks), 256, 0, ctx->stream>>>(
        reinterpret_cast<const double2 *const *>(dtab + zs.o_hb), reinterpret_cast<const int *>(dtab + zs.o_bk),
        reinterpret_cast<const int *>(dtab + zs.o_ba), reinterpret_cast<const long long *>(dtab + zs.o_br),
        reinterpret_cast<const int *>(dtab + zs.o_nb), nLMP, nlmp, zs.Kh, zs.RA,
        reinterpret_cast<__nv_bfloat16 *>(dscr + zs.s_A), reinterpret_cast<int *>(dscr + zs.s_ae));
    ak_slices_kernel<<<dim3(grid_rows(zs.npairs_pad, 8), (unsigned)na), 256, 0, ctx->stream>>>(
        reinterpret_cast<const double2 *const *>(dtab + zs.o_ha), reinterpret_cast<const int *>(dtab + zs.o_pk2),
        reinterpret_cast<const int *>(dtab + zs.o_pm), zs.npairs_a, zs.npairs_pad,
        reinterpret_cast<const long long *>(dtab + zs.o_br0), na, nlmp, zs.Kh, zs.RB,
        reinterpret_cast<__nv_bfloat16 *>(dscr + zs.s_B), reinterpret_cast<int *>(dscr + zs.s_be));
    if (nlaunch) *nlaunch += 2;
    return cuda_check(ctx, cudaGetLastError(), "muffin-tin product slices");
}

int zmt_tc_plan_batch(hfx_ctx *ctx, const ZmtPlan &zs, const std::vector<PairDesc> &pairs, long long RSc, HostArena &tab,
                      ZmtBatch &zb) {
    zb = ZmtBatch();
    if (!zs.ok) return HFX_OK;
    const int nk = ctx->nk, na = ctx->sys.n_atoms;
    const int *M = ctx->sys.mesh;
    const int npp = (int)(zs.RB / 2);
    // output column offsets per (k, pair) and phases e^{-i q.tau_a} per (k, a, k')
    std::vector<long long> coloff((size_t)nk * npp, -1);
    std::vector<float4> phase((size_t)nk * na * nk, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    std::vector<char> kin(nk, 0);
    for (const PairDesc &pr : pairs) {
        if (pr.no == 0) continue;
        kin[pr.ik] = 1;
        int j0 = pr.iq / (M[1] * M[2]), j1 = (pr.iq / M[2]) % M[1], j2 = pr.iq % M[2];
        for (int a = 0; a < na; ++a) {
            const double *tau = ctx->pos.data() + 3 * a;
            double ph = 2.0 * M_PI * ((double)j0 / M[0] * tau[0] + (double)j1 / M[1] * tau[1] + (double)j2 / M[2] * tau[2]);
            // split into FP32 pairs: hi = fl(x), lo = fl(x - hi)
            const double fr = std::cos(ph), fi = -std::sin(ph);
            const float frh = (float)fr, fih = (float)fi;
            phase[((size_t)pr.ik * na + a) * nk + pr.ikp] =
                make_float4(frh, (float)(fr - (double)frh), fih, (float)(fi - (double)fih));
            for (int m = 0; m < pr.no; ++m) {
                int ip = zs.kbase[pr.ikp] + m;
                coloff[(size_t)pr.ik * npp + (size_t)a * zs.npairs_pad + ip] = (pr.col0 + (long long)m * pr.nb) * RSc;
            }
        }
    }
    std::vector<CgTile> tiles;
    const int nchunk = 2 * zs.Kh / CG_KC;
    for (auto &bk : zs.blocks) {
        int k = bk.first, a = bk.second;
        if (!kin[k]) continue;
        long long r0 = zs.blk_row0[(size_t)k * na + a], rows = zs.blk_rows[(size_t)k * na + a];
        for (int tb = 0; tb < zs.npairs_pad / (CG_BN / 2); ++tb) {
            bool any = false;
            for (int j = 0; j < CG_BN / 2 && !any; ++j)
                any = coloff[(size_t)k * npp + (size_t)a * zs.npairs_pad + tb * (CG_BN / 2) + j] >= 0;
            if (!any) continue;
            for (long long ta = 0; ta < rows; ta += CG_BM)
                tiles.push_back(CgTile{(int)(r0 + ta), (int)((long long)a * 2 * zs.npairs_pad + tb * CG_BN), k,
                                       (k * na + a) * nk, nchunk, 0});
        }
    }
    if (tiles.empty()) return HFX_OK;
    zb.o_co = tab.put(coloff);
    zb.o_ph = tab.put(phase);
    zb.o_ti = tab.put(tiles);
    zb.ntiles = (int)tiles.size();
    zb.ok = true;
    return HFX_OK;
}

int zmt_tc_run_batch(hfx_ctx *ctx, const ZmtPlan &zs, const ZmtBatch &zb, const char *dtab, char *dscr, double2 *d_Z,
                     int *nlaunch) {
    if (!zs.ok || !zb.ok) return HFX_OK;
    CgParams p{};
    p.tiles = reinterpret_cast<const CgTile *>(dtab + zb.o_ti);
    p.ntiles = zb.ntiles;
    p.aexp = reinterpret_cast<const int *>(dscr + zs.s_ae);
    p.bexp = reinterpret_cast<const int *>(dscr + zs.s_be);
    p.rowoff = reinterpret_cast<const long long *>(dtab + zs.o_ro);
    p.coloff = reinterpret_cast<const long long *>(dtab + zb.o_co);
    p.col_gstride = zs.RB / 2;
    p.phase = reinterpret_cast<const float4 *>(dtab + zb.o_ph);
    p.pkey = reinterpret_cast<const int *>(dtab + zs.o_pk);
    p.out = d_Z;
    if (nlaunch) *nlaunch += 1;
    return launch_cgemm(ctx, reinterpret_cast<const __nv_bfloat16 *>(dscr + zs.s_A), zs.RA,
                        reinterpret_cast<const __nv_bfloat16 *>(dscr + zs.s_B), zs.RB, 2 * zs.Kh, p);
}

}  // namespace hfx
