// k_stage1.cu -- projection vectors Z_q[I,m,n] = < M_I^q phi_{m,k-q} | phi_{n,k} >
// (Sec. III.B, Eq. vec-mat-vec), templated on the arithmetic type (float for
// the split-precision build, double for the FP64 build).
//
//   MT part (per k, then per pair):
//     B_k[a][LM][i][lmp][n] = sum_P T_{aL}[i][P] sum_{l'p'} G(LM; lm; l', m+M) R^a_{LP;lp;l'p'} A^a_{l',m+M,p'}(n,k)
//     Z[(a,LM,i), m, n]     = e^{-i q.R_a} sum_{lmp} conj(A^a_{lmp}(m,k')) B_k[a][LM][i][lmp][n]
//   interstitial part (per k, then per pair):
//     T_n(K)     = sum_{G2 in k} Theta_{K - G2} c_{G2}(n,k)        (step-function weighted wave function)
//     Z[G, m, n] = Omega^{-1/2} sum_{G1 in k'} conj(c_{G1}(m,k')) T_n(G + G1 - G0),  G0 = k - q - k'
//
// Output Zc[col][row]: column col = pair col0 + m*nb + n, row in the permuted
// MPB order [mu=0 | mu!=0 | IPW] (sparse) or the original order (dense).
#include <algorithm>

#include "hfx_internal.cuh"

namespace hfx {

namespace {

constexpr double kPi = 3.14159265358979323846;

template <typename R> __device__ __forceinline__ typename C2<R>::T ld_c(const double2 &x) {
    typename C2<R>::T r;
    r.x = (R)x.x;
    r.y = (R)x.y;
    return r;
}

// ------------------------------------------------------------- Theta psi
template <typename R>
__global__ void thetapsi_kernel(const double2 *__restrict__ theta, int dlo0, int dlo1, int dlo2, int dd1, int dd2,
                                int tlo0, int tlo1, int tlo2, int td0, int td1, int td2,
                                const double2 *__restrict__ c, const int *__restrict__ G, int nb, int npw,
                                typename C2<R>::T *__restrict__ out) {
    using V = typename C2<R>::T;
    constexpr int NCH = 8, GT = 128;
    __shared__ V cs[NCH][GT];
    __shared__ int offs[GT];
    long long box = (long long)td0 * td1 * td2;
    long long K = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int n0 = blockIdx.y * NCH;
    int kz = 0, ky = 0, kx = 0;
    long long dbase = 0;
    if (K < box) {
        kz = (int)(K % td2);
        ky = (int)((K / td2) % td1);
        kx = (int)(K / ((long long)td1 * td2));
        // linear index of (K - dlo) in the difference box; the G2 shift is subtracted below
        dbase = ((long long)(tlo0 + kx - dlo0) * dd1 + (tlo1 + ky - dlo1)) * dd2 + (tlo2 + kz - dlo2);
    }
    V acc[NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) acc[j] = cmk<V>(0, 0);
    for (int g0 = 0; g0 < npw; g0 += GT) {
        int gn = min(GT, npw - g0);
        __syncthreads();
        for (int t = threadIdx.x; t < gn; t += blockDim.x) {
            const int *g = G + 3 * (g0 + t);
            offs[t] = (g[0] * dd1 + g[1]) * dd2 + g[2];
        }
        for (int t = threadIdx.x; t < NCH * GT; t += blockDim.x) {
            int j = t / GT, gi = t % GT;
            int n = n0 + j;
            cs[j][gi] = (n < nb && gi < gn) ? ld_c<R>(c[(size_t)n * npw + g0 + gi]) : cmk<V>(0, 0);
        }
        __syncthreads();
        if (K < box) {
            for (int gi = 0; gi < gn; ++gi) {
                V th = ld_c<R>(theta[dbase - offs[gi]]);
#pragma unroll
                for (int j = 0; j < NCH; ++j) acc[j] = cfma(th, cs[j][gi], acc[j]);
            }
        }
    }
    if (K < box) {
#pragma unroll
        for (int j = 0; j < NCH; ++j)
            if (n0 + j < nb) out[(size_t)(n0 + j) * box + K] = acc[j];
    }
}

// ------------------------------------------------------------- B_k
template <typename R>
__global__ void bmat_kernel(const double2 *__restrict__ A, const double *__restrict__ Rr, const double *__restrict__ T,
                            const double *__restrict__ gaunt, int n_atoms, int lmax, int Lmax, int P, int nb,
                            int use_T, typename C2<R>::T *__restrict__ Bk) {
    using V = typename C2<R>::T;
    int nlm = (lmax + 1) * (lmax + 1), nLM = (Lmax + 1) * (Lmax + 1), nlmp = 2 * nlm, nlp = 2 * (lmax + 1);
    long long total = (long long)n_atoms * nLM * nlmp * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int n = (int)(e % nb);
        int lmp = (int)((e / nb) % nlmp);
        int LM = (int)((e / ((long long)nb * nlmp)) % nLM);
        int a = (int)(e / ((long long)nb * nlmp * nLM));
        int lm = lmp >> 1, p = lmp & 1;
        int l = (int)floor(sqrt((double)lm) + 1e-9), m = lm - l * l - l;
        int L = (int)floor(sqrt((double)LM) + 1e-9), M = LM - L * L - L;
        double2 bp[kMaxP];
        for (int s = 0; s < P; ++s) bp[s] = make_double2(0.0, 0.0);
        const double2 *An = A + ((size_t)n * n_atoms + a) * nlmp;
        for (int l2 = 0; l2 <= lmax; ++l2) {
            int m2 = m + M;
            if (m2 < -l2 || m2 > l2) continue;
            double g = gaunt[((size_t)LM * nlm + lm) * (lmax + 1) + l2];
            if (g == 0.0) continue;
            for (int p2 = 0; p2 < 2; ++p2) {
                double2 av = An[2 * (l2 * l2 + l2 + m2) + p2];
                for (int s = 0; s < P; ++s) {
                    double r = Rr[(((size_t)a * (Lmax + 1) + L) * P + s) * nlp * nlp + (2 * l + p) * nlp + 2 * l2 + p2];
                    bp[s].x += g * r * av.x;
                    bp[s].y += g * r * av.y;
                }
            }
        }
        const double *Ta = T + ((size_t)a * (Lmax + 1) + L) * P * P;
        for (int i = 0; i < P; ++i) {
            double2 o;
            if (use_T) {
                o = make_double2(0.0, 0.0);
                for (int s = 0; s < P; ++s) {
                    o.x += Ta[i * P + s] * bp[s].x;
                    o.y += Ta[i * P + s] * bp[s].y;
                }
            } else {
                o = bp[i];
            }
            Bk[((((size_t)a * nLM + LM) * P + i) * nlmp + lmp) * nb + n] = ld_c<R>(o);
        }
    }
}

// ------------------------------------------------------------- Z^MT
// One block per (pair, atom); A_{k'} of the atom in shared memory.
template <typename R>
__global__ void zmt_kernel(const PairDesc *__restrict__ pairs, const QDesc *__restrict__ qd,
                           typename C2<R>::T *const *__restrict__ Bk, const double2 *const *__restrict__ Ak,
                           const double *__restrict__ posf, int m0, int m1, int m2, int n_atoms, int nLM, int P,
                           int nlmp, int N0, int sparse, typename C2<R>::T *__restrict__ Z, long long RSc) {
    using V = typename C2<R>::T;
    extern __shared__ unsigned char smem_raw[];
    V *As = reinterpret_cast<V *>(smem_raw);  // [no][nlmp]
    const PairDesc pr = pairs[blockIdx.x];
    int a = blockIdx.y;
    int nb = pr.nb, no = pr.no;
    const double2 *Akp = Ak[pr.ikp];
    for (int t = threadIdx.x; t < no * nlmp; t += blockDim.x) {
        int m = t / nlmp, j = t % nlmp;
        double2 v = Akp[((size_t)m * n_atoms + a) * nlmp + j];
        As[t] = ld_c<R>(v);
    }
    __syncthreads();
    int j2 = pr.iq % m2, j1 = (pr.iq / m2) % m1, j0 = pr.iq / (m1 * m2);
    double ph = 2.0 * kPi * ((double)j0 / m0 * posf[3 * a] + (double)j1 / m1 * posf[3 * a + 1] +
                             (double)j2 / m2 * posf[3 * a + 2]);
    double sp, cp;
    sincos(ph, &sp, &cp);
    V phase = cmk<V>((R)cp, (R)(-sp));
    const V *B = Bk[pr.ik];
    int nch = n_atoms * nLM;
    int rows = nLM * P;
    constexpr int MCH = 8;
    for (int t = threadIdx.x; t < rows * nb; t += blockDim.x) {
        int n = t % nb, r = t / nb;
        int LM = r / P, i = r % P;
        int ch = a * nLM + LM;
        int row = sparse ? (i == 0 ? N0 + ch : ch * (P - 1) + i - 1) : ch * P + i;
        const V *Bp = B + (((size_t)ch * P + i) * nlmp) * nb + n;
        for (int mb = 0; mb < no; mb += MCH) {
            V acc[MCH];
#pragma unroll
            for (int j = 0; j < MCH; ++j) acc[j] = cmk<V>(0, 0);
            for (int lmp = 0; lmp < nlmp; ++lmp) {
                V b = Bp[(size_t)lmp * nb];
#pragma unroll
                for (int j = 0; j < MCH; ++j)
                    if (mb + j < no) acc[j] = cfma_conj(As[(mb + j) * nlmp + lmp], b, acc[j]);
            }
#pragma unroll
            for (int j = 0; j < MCH; ++j)
                if (mb + j < no) {
                    long long col = pr.col0 + (long long)(mb + j) * nb + n;
                    Z[col * RSc + row] = cmul(phase, acc[j]);
                }
        }
    }
    (void)nch;
    (void)qd;
}

// ------------------------------------------------------------- Z^IPW
// One block per (k, n); T_n of k stays in shared memory (TSM) or is read from
// global memory, and the block walks over every q of the batch.
template <typename R, bool TSM>
__global__ void zipw_kernel(const PairDesc *__restrict__ pairs, const int *__restrict__ kpairs /* [nk][nq] */,
                            const QDesc *__restrict__ qd, int nq, typename C2<R>::T *const *__restrict__ Tk,
                            int tlo0, int tlo1, int tlo2, int td1, int td2, long long box,
                            const double2 *const *__restrict__ ck, const int *const *__restrict__ Gk,
                            const int *__restrict__ npw_k, const int *const *__restrict__ Gaux,
                            const int *__restrict__ nb_k, R rs_omega, int rowbase_ipw,
                            typename C2<R>::T *__restrict__ Z, long long RSc, int cmax) {
    using V = typename C2<R>::T;
    constexpr int MCH = (sizeof(R) == 4) ? 8 : 4;
    extern __shared__ unsigned char smem_raw[];
    int n = blockIdx.x, ik = blockIdx.y;
    if (n >= nb_k[ik]) return;
    int nb = nb_k[ik];
    V *Ts = reinterpret_cast<V *>(smem_raw);
    V *cs = Ts + (TSM ? box : 0);                         // [MCH][cmax]
    int *offs = reinterpret_cast<int *>(cs + (size_t)MCH * cmax);  // [cmax]
    const V *Tn = Tk[ik] + (size_t)n * box;
    if (TSM) {
        for (long long t = threadIdx.x; t < box; t += blockDim.x) Ts[t] = Tn[t];
    }
    const V *Tuse = TSM ? Ts : Tn;
    for (int qs = 0; qs < nq; ++qs) {
        int pi = kpairs[(size_t)ik * nq + qs];
        if (pi < 0) continue;
        const PairDesc pr = pairs[pi];
        const QDesc q = qd[qs];
        int ikp = pr.ikp, no = pr.no;
        int npw = npw_k[ikp];
        const double2 *cp = ck[ikp];
        const int *G1 = Gk[ikp];
        const int *Ga = Gaux[q.iq];
        for (int mb = 0; mb < no; mb += MCH) {
            __syncthreads();
            for (int t = threadIdx.x; t < npw; t += blockDim.x) {
                offs[t] = (G1[3 * t] * td1 + G1[3 * t + 1]) * td2 + G1[3 * t + 2];
            }
            for (int t = threadIdx.x; t < MCH * npw; t += blockDim.x) {
                int j = t / npw, gi = t % npw;
                int m = mb + j;
                cs[(size_t)j * cmax + gi] = (m < no) ? ld_c<R>(cp[(size_t)m * npw + gi]) : cmk<V>(0, 0);
            }
            __syncthreads();
            for (int g = threadIdx.x; g < q.nipw; g += blockDim.x) {
                // index of K = G + G1 - G0 in the T box is base(G - G0) + offs(G1)
                long long base = ((long long)(Ga[3 * g] - pr.g0[0] - tlo0) * td1 + (Ga[3 * g + 1] - pr.g0[1] - tlo1)) * td2 +
                                 (Ga[3 * g + 2] - pr.g0[2] - tlo2);
                V acc[MCH];
#pragma unroll
                for (int j = 0; j < MCH; ++j) acc[j] = cmk<V>(0, 0);
                for (int gi = 0; gi < npw; ++gi) {
                    V t = Tuse[base + offs[gi]];
#pragma unroll
                    for (int j = 0; j < MCH; ++j) acc[j] = cfma_conj(cs[(size_t)j * cmax + gi], t, acc[j]);
                }
#pragma unroll
                for (int j = 0; j < MCH; ++j) {
                    int m = mb + j;
                    if (m < no) {
                        long long col = pr.col0 + (long long)m * nb + n;
                        V o = acc[j];
                        o.x *= rs_omega;
                        o.y *= rs_omega;
                        Z[col * RSc + rowbase_ipw + g] = o;
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------- overrides
// Z supplied by the caller in the original order -> permuted, transformed.
template <typename R>
__global__ void override_kernel(const double2 *__restrict__ U, PairDesc pr, int naux, const double *__restrict__ T,
                                int n_atoms, int Lmax, int P, int N0, int sparse, typename C2<R>::T *__restrict__ Z,
                                long long RSc, int nmt) {
    int nLM = (Lmax + 1) * (Lmax + 1), nch = n_atoms * nLM;
    long long total = (long long)naux * pr.no * pr.nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int n = (int)(e % pr.nb), m = (int)((e / pr.nb) % pr.no), p = (int)(e / ((long long)pr.nb * pr.no));
        double2 val = make_double2(0.0, 0.0);
        size_t mn = (size_t)m * pr.nb + n;
        size_t stride = (size_t)pr.no * pr.nb;
        if (!sparse) {
            val = U[(size_t)p * stride + mn];
        } else if (p >= N0 + nch) {
            val = U[(size_t)(nmt + p - N0 - nch) * stride + mn];
        } else {
            int ch, i;
            if (p < N0) { ch = p / (P - 1); i = 1 + p % (P - 1); }
            else { ch = p - N0; i = 0; }
            int a = ch / nLM, L = (int)floor(sqrt((double)(ch % nLM)) + 1e-9);
            const double *Tr = T + (((size_t)a * (Lmax + 1) + L) * P + i) * P;
            for (int s = 0; s < P; ++s) {
                double2 u = U[(size_t)(ch * P + s) * stride + mn];
                val.x += Tr[s] * u.x;
                val.y += Tr[s] * u.y;
            }
        }
        long long col = pr.col0 + (long long)m * pr.nb + n;
        Z[col * RSc + p] = ld_c<R>(val);
    }
}

// Zc (permuted, transformed) -> original order, FP64 [naux][no][nb].
template <typename R>
__global__ void unpermute_kernel(const typename C2<R>::T *__restrict__ Z, PairDesc pr, int naux,
                                 const double *__restrict__ T, int n_atoms, int Lmax, int P, int N0, int sparse,
                                 long long RSc, int nmt, double2 *__restrict__ out) {
    int nLM = (Lmax + 1) * (Lmax + 1), nch = n_atoms * nLM;
    long long total = (long long)naux * pr.no * pr.nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int n = (int)(e % pr.nb), m = (int)((e / pr.nb) % pr.no), I = (int)(e / ((long long)pr.nb * pr.no));
        long long col = pr.col0 + (long long)m * pr.nb + n;
        const typename C2<R>::T *zc = Z + col * RSc;
        double2 val = make_double2(0.0, 0.0);
        if (!sparse) {
            val = make_double2((double)zc[I].x, (double)zc[I].y);
        } else if (I >= nmt) {
            auto z = zc[N0 + nch + (I - nmt)];
            val = make_double2((double)z.x, (double)z.y);
        } else {
            int ch = I / P, s = I % P;
            int a = ch / nLM, L = (int)floor(sqrt((double)(ch % nLM)) + 1e-9);
            const double *Ta = T + ((size_t)a * (Lmax + 1) + L) * P * P;
            for (int i = 0; i < P; ++i) {  // Z = T^T Z_t
                int row = (i == 0) ? N0 + ch : ch * (P - 1) + i - 1;
                auto z = zc[row];
                val.x += Ta[i * P + s] * (double)z.x;
                val.y += Ta[i * P + s] * (double)z.y;
            }
        }
        out[e] = val;
    }
}

// Sec. III.D, Eqs. (sym MT functions): Z' = S^H Z, Z'_I = sum_J conj(S_JI) Z_J.
// For a pair of rows (the first and second function of one symmetrized pair,
// s = (-1)^(L+M)):  first' = (z1 + s z2)/sqrt2,  second' = -i (z1 - s z2)/sqrt2;
// a lone row (M = 0, odd L, atom at an inversion centre) becomes -i z.
template <typename V>
__global__ void sym_rows_kernel(V *__restrict__ Z, long long RSc, long long ncols, const SymOp *__restrict__ ops,
                                int nops) {
    const double h = 0.70710678118654752440;
    const long long total = ncols * nops;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long col = e / nops;
        const SymOp op = ops[e % nops];
        V *z = Z + col * RSc;
        const V a = z[op.r1];
        if (op.kind == 2) {
            z[op.r1] = ld_c<decltype(a.x)>(make_double2((double)a.y, -(double)a.x));
            continue;
        }
        const V b = z[op.r2];
        const double sg = op.kind == 0 ? 1.0 : -1.0;
        const double fx = ((double)a.x + sg * b.x) * h, fy = ((double)a.y + sg * b.y) * h;
        const double dx = ((double)a.x - sg * b.x) * h, dy = ((double)a.y - sg * b.y) * h;
        z[op.r1] = ld_c<decltype(a.x)>(make_double2(fx, fy));
        z[op.r2] = ld_c<decltype(a.x)>(make_double2(dy, -dx));
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 32) g = 152LL * 32;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// The row operations of Z' = S^H Z in the batch row layout: MT function
// (a, L, M, i) of the transformed (sparse) or original (dense) order sits in row
// N0 + ch (sparse, i = 0), ch (P - 1) + i - 1 (sparse, i >= 1) or ch P + i
// (dense), ch = a (Lmax+1)^2 + L^2 + L + M.  Partner channels share their
// multipole transform (equal multipoles), so the pairing acts index by index.
std::vector<SymOp> sym_row_ops(const hfx_ctx *ctx, int N0, int sparse) {
    std::vector<SymOp> ops;
    const int P = ctx->P, Lmax = ctx->sys.Lmax, nLM = ctx->nLM;
    auto row = [&](int a, int L, int M, int i) {
        const int ch = a * nLM + L * L + L + M;
        if (!sparse) return ch * P + i;
        return i == 0 ? N0 + ch : ch * (P - 1) + i - 1;
    };
    for (int a = 0; a < ctx->sys.n_atoms; ++a) {
        const int b = ctx->partner[a];
        for (int L = 0; L <= Lmax; ++L)
            for (int M = -L; M <= L; ++M) {
                const int kind = ((L + M) % 2 == 0) ? 0 : 1;
                for (int i = 0; i < P; ++i) {
                    if (a == b && M == 0) {
                        if (L % 2) ops.push_back(SymOp{row(a, L, 0, i), -1, 2, 0});
                    } else if (a < b || (a == b && M < 0)) {
                        ops.push_back(SymOp{row(a, L, M, i), row(b, L, -M, i), kind, 0});
                    }
                }
            }
    }
    std::sort(ops.begin(), ops.end(), [](const SymOp &x, const SymOp &y) { return x.r1 < y.r1; });
    return ops;
}

template <typename V>
void launch_sym_rows(V *d_Z, long long RSc, long long ncols, const SymOp *d_ops, int nops, cudaStream_t st) {
    if (nops == 0 || ncols == 0) return;
    sym_rows_kernel<V><<<grid_for(ncols * nops, 256), 256, 0, st>>>(d_Z, RSc, ncols, d_ops, nops);
}
template void launch_sym_rows<float2>(float2 *, long long, long long, const SymOp *, int, cudaStream_t);
template void launch_sym_rows<double2>(double2 *, long long, long long, const SymOp *, int, cudaStream_t);

template <typename R>
void launch_thetapsi(const double2 *d_theta, const int dlo[3], const int ddim[3], const int tlo[3], const int tdim[3],
                     const double2 *d_c, const int *d_G, int nb, int npw, typename C2<R>::T *d_out,
                     cudaStream_t st) {
    long long box = (long long)tdim[0] * tdim[1] * tdim[2];
    dim3 grid((unsigned)((box + 127) / 128), (unsigned)((nb + 7) / 8));
    thetapsi_kernel<R><<<grid, 128, 0, st>>>(d_theta, dlo[0], dlo[1], dlo[2], ddim[1], ddim[2], tlo[0], tlo[1],
                                             tlo[2], tdim[0], tdim[1], tdim[2], d_c, d_G, nb, npw, d_out);
}

template <typename R>
void launch_bmat(const double2 *d_A, const double *d_R, const double *d_T, const double *d_gaunt, int n_atoms,
                 int lmax, int Lmax, int P, int nb, int use_T, typename C2<R>::T *d_B, cudaStream_t st) {
    long long total = (long long)n_atoms * (Lmax + 1) * (Lmax + 1) * 2 * (lmax + 1) * (lmax + 1) * nb;
    bmat_kernel<R><<<grid_for(total, 128), 128, 0, st>>>(d_A, d_R, d_T, d_gaunt, n_atoms, lmax, Lmax, P, nb, use_T,
                                                         d_B);
}

template <typename R>
void launch_zmt(const PairDesc *d_pairs, int npairs, const QDesc *d_q, typename C2<R>::T *const *d_Bk,
                const double2 *const *d_Ak, const double *d_posf, const int mesh[3], int n_atoms, int nLM, int P,
                int nlmp, int N0, int sparse, int no_max, typename C2<R>::T *d_Z, long long RSc, cudaStream_t st) {
    if (npairs == 0) return;
    size_t sm = (size_t)no_max * nlmp * sizeof(typename C2<R>::T);
    if (sm > 48 * 1024) cudaFuncSetAttribute(zmt_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((unsigned)npairs, (unsigned)n_atoms);
    zmt_kernel<R><<<grid, 256, sm, st>>>(d_pairs, d_q, d_Bk, d_Ak, d_posf, mesh[0], mesh[1], mesh[2], n_atoms, nLM,
                                         P, nlmp, N0, sparse, d_Z, RSc);
}

template <typename R>
int launch_zipw(const PairDesc *d_pairs, const int *d_kpairs, int nk, int nb_max, const QDesc *d_q, int nq,
                typename C2<R>::T *const *d_Tk, const int tlo[3], const int tdim[3], const double2 *const *d_ck,
                const int *const *d_Gk, const int *d_npw, int npw_max, const int *const *d_Gaux, const int *d_nb_k,
                double omega, int rowbase_ipw, typename C2<R>::T *d_Z, long long RSc, cudaStream_t st) {
    using V = typename C2<R>::T;
    constexpr int MCH = (sizeof(R) == 4) ? 8 : 4;
    long long box = (long long)tdim[0] * tdim[1] * tdim[2];
    int cmax = npw_max;
    size_t small = (size_t)MCH * cmax * sizeof(V) + (size_t)cmax * sizeof(int);
    size_t big = small + (size_t)box * sizeof(V);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, 0);
    dim3 grid((unsigned)nb_max, (unsigned)nk);
    R rs = (R)(1.0 / sqrt(omega));
    if (big <= (size_t)maxsm) {
        cudaFuncSetAttribute(zipw_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big);
        zipw_kernel<R, true><<<grid, 256, big, st>>>(d_pairs, d_kpairs, d_q, nq, d_Tk, tlo[0], tlo[1], tlo[2],
                                                     tdim[1], tdim[2], box, d_ck, d_Gk, d_npw, d_Gaux, d_nb_k, rs,
                                                     rowbase_ipw, d_Z, RSc, cmax);
    } else {
        if (small > (size_t)maxsm) return HFX_EUNSUPPORTED;
        cudaFuncSetAttribute(zipw_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)small);
        zipw_kernel<R, false><<<grid, 256, small, st>>>(d_pairs, d_kpairs, d_q, nq, d_Tk, tlo[0], tlo[1], tlo[2],
                                                        tdim[1], tdim[2], box, d_ck, d_Gk, d_npw, d_Gaux, d_nb_k, rs,
                                                        rowbase_ipw, d_Z, RSc, cmax);
    }
    return HFX_OK;
}

template <typename R>
void launch_override(const double2 *d_user, const PairDesc &pr, int naux, const double *d_T, int n_atoms, int Lmax,
                     int P, int N0, int sparse, typename C2<R>::T *d_Z, long long RSc, int nmt, cudaStream_t st) {
    long long total = (long long)naux * pr.no * pr.nb;
    override_kernel<R><<<grid_for(total, 256), 256, 0, st>>>(d_user, pr, naux, d_T, n_atoms, Lmax, P, N0, sparse,
                                                             d_Z, RSc, nmt);
}

template <typename R>
void launch_unpermute(const typename C2<R>::T *d_Z, const PairDesc &pr, int naux, const double *d_T, int n_atoms,
                      int Lmax, int P, int N0, int sparse, long long RSc, int nmt, double2 *d_out, cudaStream_t st) {
    long long total = (long long)naux * pr.no * pr.nb;
    unpermute_kernel<R><<<grid_for(total, 256), 256, 0, st>>>(d_Z, pr, naux, d_T, n_atoms, Lmax, P, N0, sparse, RSc,
                                                              nmt, d_out);
}

#define HFX_INST(R)                                                                                                  \
    template void launch_thetapsi<R>(const double2 *, const int *, const int *, const int *, const int *,            \
                                     const double2 *, const int *, int, int, C2<R>::T *, cudaStream_t);              \
    template void launch_bmat<R>(const double2 *, const double *, const double *, const double *, int, int, int,    \
                                 int, int, int, C2<R>::T *, cudaStream_t);                                           \
    template void launch_zmt<R>(const PairDesc *, int, const QDesc *, C2<R>::T *const *, const double2 *const *,    \
                                const double *, const int *, int, int, int, int, int, int, int, C2<R>::T *,         \
                                long long, cudaStream_t);                                                            \
    template int launch_zipw<R>(const PairDesc *, const int *, int, int, const QDesc *, int, C2<R>::T *const *,     \
                                const int *, const int *, const double2 *const *, const int *const *, const int *,  \
                                int, const int *const *, const int *, double, int, C2<R>::T *, long long,           \
                                cudaStream_t);                                                                       \
    template void launch_override<R>(const double2 *, const PairDesc &, int, const double *, int, int, int, int,    \
                                     int, C2<R>::T *, long long, int, cudaStream_t);                                 \
    template void launch_unpermute<R>(const C2<R>::T *, const PairDesc &, int, const double *, int, int, int, int,  \
                                      int, long long, int, double2 *, cudaStream_t);

HFX_INST(float)
HFX_INST(double)

}  // namespace hfx
