// k_contract64.cu -- the plain FP64 contraction (the "plain FP64 GPU" build):
// Y = v_t Z (dense block and mu=0 blocks of Fig. 1) and the per-pair
// V partial P[n][n'] = sum_m sum_I conj(Z[I,m,n]) Y[I,m,n'] (Eq. vec-mat-vec),
// with DFMA on the CUDA cores.
#include "hfx_internal.cuh"

namespace hfx {

namespace {

constexpr int TM = 64, TN = 64, TK = 8;

// Batched complex GEMM, C = op(A) B, K = K1 * K2 split into two strides.
__global__ void __launch_bounds__(256) zgemm64_kernel(const ZGemmBatch *__restrict__ batches) {
    const ZGemmBatch b = batches[blockIdx.z];
    int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
    if (i0 >= b.M || j0 >= b.N) return;
    __shared__ double2 As[TK][TM + 1];
    __shared__ double2 Bs[TK][TN + 1];
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
    long long K = (long long)b.K1 * b.K2;
    for (long long k0 = 0; k0 < K; k0 += TK) {
        for (int t = threadIdx.x; t < TK * TM; t += 256) {
            int kk = t / TM, r = t % TM;
            long long k = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (k < K && i0 + r < b.M) {
                long long k1 = k / b.K2, k2 = k % b.K2;
                v = b.A[(i0 + r) * b.sAi + k1 * b.sAk1 + k2 * b.sAk2];
                if (b.conjA) v.y = -v.y;
            }
            As[kk][r] = v;
        }
        for (int t = threadIdx.x; t < TK * TN; t += 256) {
            int kk = t / TN, c = t % TN;
            long long k = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (k < K && j0 + c < b.N) {
                long long k1 = k / b.K2, k2 = k % b.K2;
                v = b.B[k1 * b.sBk1 + k2 * b.sBk2 + (j0 + c) * b.sBj];
            }
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            double2 a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
            if (r < b.M && c < b.N) b.C[r * b.sCi + c * b.sCj] = acc[i][j];
        }
}

// Y rows of the mu=0 functions: per channel, the (P-1) x P block times the
// channel's [mu!=0, mu=0...] rows of Z (Fig. 1 on-site blocks).
__global__ void block64_kernel(const QDesc *__restrict__ qd, const double2 *const *__restrict__ VB,
                               const double2 *__restrict__ Z, double2 *__restrict__ Y, long long RSc, int nch, int P,
                               int N0) {
    const QDesc q = qd[blockIdx.y];
    const double2 *vb = VB[blockIdx.y];
    long long total = q.ncols * N0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int u = (int)(e % N0);
        long long col = q.colbase + e / N0;
        int ch = u / (P - 1), i = u % (P - 1);
        const double2 *z = Z + col * RSc;
        const double2 *row = vb + ((size_t)ch * (P - 1) + i) * P;
        double2 acc = cmul(row[0], z[N0 + ch]);
        for (int s = 1; s < P; ++s) acc = cfma(row[s], z[ch * (P - 1) + s - 1], acc);
        Y[col * RSc + u] = acc;
    }
}

}  // namespace

void launch_zgemm64(const ZGemmBatch *d_b, int nbatch, int maxM, int maxN, cudaStream_t st) {
    if (nbatch == 0) return;
    dim3 grid((unsigned)((maxN + TN - 1) / TN), (unsigned)((maxM + TM - 1) / TM), (unsigned)nbatch);
    zgemm64_kernel<<<grid, 256, 0, st>>>(d_b);
}

void launch_block64(const QDesc *d_q, int nq, const double2 *const *d_VB, const double2 *d_Z, double2 *d_Y,
                    long long RSc, int nch, int P, int N0, long long maxcols, cudaStream_t st) {
    if (N0 == 0 || nq == 0) return;
    long long per = maxcols * N0;
    long long g = (per + 255) / 256;
    if (g > 4096) g = 4096;
    dim3 grid((unsigned)g, (unsigned)nq);
    block64_kernel<<<grid, 256, 0, st>>>(d_q, d_VB, d_Z, d_Y, RSc, nch, P, N0);
}

}  // namespace hfx
