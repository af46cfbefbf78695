// k_finish.cu -- FP64 Brillouin-zone sum over q, the q->0 term of
// Eq. (div final) and the exchange energy, all in FP64.
#include "hfx_internal.cuh"

namespace hfx {

namespace {

// Vacc[k] += sum_{pairs of k in this batch, ascending q} P_pair, where the
// tensor-core tiles (raw_format 1) hold P' = Z^H U Z and P_pair = P' + P'^H.
__global__ void reduce_pairs_kernel(const PairDesc *__restrict__ pairs, const int *__restrict__ kstart,
                                    const int *__restrict__ klist_pairs, const int *__restrict__ klist,
                                    const double *__restrict__ praw, const long long *__restrict__ praw_off, int NB,
                                    int raw_format, double2 *const *__restrict__ vacc, const int *__restrict__ nb_k) {
    int slot = blockIdx.y;
    int ik = klist[slot];
    int nb = nb_k[ik];
    int p0 = kstart[slot], p1 = kstart[slot + 1];
    double2 *V = vacc[ik];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nb * nb; e += gridDim.x * blockDim.x) {
        int n = e / nb, n2 = e % nb;
        double2 acc = V[e];
        for (int t = p0; t < p1; ++t) {
            int pi = klist_pairs[t];
            const double *P = praw + praw_off[pi];
            if (raw_format == 0) {
                const double2 *Pc = reinterpret_cast<const double2 *>(P);
                double2 v = Pc[(size_t)n * nb + n2];
                acc.x += v.x;
                acc.y += v.y;
            } else {
                // real-embedded tiles of P' = Z^H U Z; the pair's term is P' + P'^H
                int nblk = (nb + NB - 1) / NB;
                int bi = n / NB, a = n % NB, bj = n2 / NB, b = n2 % NB;
                int W = 2 * NB;
                const double *t0 = P + ((size_t)bi * nblk + bj) * W * W;
                const double *t1 = P + ((size_t)bj * nblk + bi) * W * W;
                double pr = t0[(size_t)a * W + b] + t0[(size_t)(NB + a) * W + NB + b];
                double pim = t0[(size_t)a * W + NB + b] - t0[(size_t)(NB + a) * W + b];
                double qr = t1[(size_t)b * W + a] + t1[(size_t)(NB + b) * W + NB + a];
                double qim = t1[(size_t)b * W + NB + a] - t1[(size_t)(NB + b) * W + a];
                acc.x += pr + qr;
                acc.y += pim - qim;
            }
        }
        V[e] = acc;
    }
    (void)pairs;
}

// V = -(1/N_k) Vacc - delta_nn' f_nk b, and E_x = (1/2)(1/N_k) sum_k sum_{n<no} Re V_nn.
__global__ void finish_kernel(double2 *const *__restrict__ vacc, double2 *const *__restrict__ Vout,
                              const int *__restrict__ nb_k, const int *__restrict__ no_k, int nk, double inv_nk,
                              double q0b, int q0_on) {
    int ik = blockIdx.y;
    int nb = nb_k[ik], no = no_k[ik];
    const double2 *A = vacc[ik];
    double2 *V = Vout[ik];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nb * nb; e += gridDim.x * blockDim.x) {
        int n = e / nb, n2 = e % nb;
        double2 a = A[e];
        double2 v = make_double2(-inv_nk * a.x, -inv_nk * a.y);
        if (q0_on && n == n2 && n < no) v.x -= q0b;
        V[e] = v;
    }
}

__global__ void energy_kernel(double2 *const *__restrict__ Vout, const int *__restrict__ nb_k,
                              const int *__restrict__ no_k, int nk, double inv_nk, double *Ex) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int ik = 0; ik < nk; ++ik) {
        int nb = nb_k[ik], no = no_k[ik];
        const double2 *V = Vout[ik];
        for (int n = threadIdx.x; n < no; n += blockDim.x) acc += V[(size_t)n * nb + n].x;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) Ex[0] = 0.5 * inv_nk * red[0];
}

}  // namespace

void launch_reduce_pairs(const PairDesc *d_pairs, const int *d_kstart, const int *d_klist_pairs, int nk_in_batch,
                         const int *d_klist, const double *d_praw, const long long *d_praw_off, int NB, int raw_format,
                         double2 *const *d_vacc, const int *d_nb_k, int nb_max, cudaStream_t st) {
    if (nk_in_batch == 0) return;
    int nx = (nb_max * nb_max + 255) / 256;
    if (nx > 64) nx = 64;
    dim3 grid((unsigned)nx, (unsigned)nk_in_batch);
    reduce_pairs_kernel<<<grid, 256, 0, st>>>(d_pairs, d_kstart, d_klist_pairs, d_klist, d_praw, d_praw_off, NB,
                                              raw_format, d_vacc, d_nb_k);
}

void launch_finish(double2 *const *d_vacc, double2 *const *d_V, const int *d_nb_k, const int *d_no_k, int nk,
                   int nb_max, double inv_nk, double q0b, int q0_on, double *d_Ex, cudaStream_t st) {
    int nx = (nb_max * nb_max + 255) / 256;
    if (nx > 64) nx = 64;
    dim3 grid((unsigned)nx, (unsigned)nk);
    finish_kernel<<<grid, 256, 0, st>>>(d_vacc, d_V, d_nb_k, d_no_k, nk, inv_nk, q0b, q0_on);
    energy_kernel<<<1, 256, 0, st>>>(d_V, d_nb_k, d_no_k, nk, inv_nk, d_Ex);
}

}  // namespace hfx
