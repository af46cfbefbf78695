// k_finish.cu -- FP64 Brillouin-zone sum over q, the q->0 term of
// Eq. (div final) and the exchange energy, all in FP64.
#include "hfx_internal.cuh"

namespace hfx {

namespace {

// Vacc[k] += sum_{pairs of k in this batch, ascending q} P_pair, where the
// tensor-core tiles (raw_format 1) hold P' = Z^H U Z and P_pair = P' + P'^H
// (raw_format 2: the real tiles of the inversion-symmetric path, Re P' only).
// With real_part (inversion symmetry, two real bands packed per column, Sec.
// III.D) only the real part is the pair's term; the imaginary part holds the
// cross products of the two bands and is dropped.
__global__ void reduce_pairs_kernel(const PairDesc *__restrict__ pairs, const int *__restrict__ kstart,
                                    const int *__restrict__ klist_pairs, const int *__restrict__ klist,
                                    const double *__restrict__ praw, const long long *__restrict__ praw_off, int NB,
                                    int raw_format, int real_part, double2 *const *__restrict__ vacc,
                                    const int *__restrict__ nb_k) {
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
                if (!real_part) acc.y += v.y;
            } else if (raw_format == 2) {
                // real tiles: Re P' in the real-real quadrant of each block
                int nblk = (nb + NB - 1) / NB;
                int bi = n / NB, a = n % NB, bj = n2 / NB, b = n2 % NB;
                int W = 2 * NB;
                acc.x += P[((size_t)bi * nblk + bj) * W * W + (size_t)a * W + b] +
                         P[((size_t)bj * nblk + bi) * W * W + (size_t)b * W + a];
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
                if (!real_part) acc.y += pim - qim;
            }
        }
        V[e] = acc;
    }
    (void)pairs;
}

// V = -(1/N_k) Vacc - delta_nn' f_nk b, and E_x = (1/2)(1/N_k) sum_k sum_{n<no} Re V_nn.
__global__ void finish_kernel(double2 *const *__restrict__ vacc, double2 *const *__restrict__ Vout,
                              const int *__restrict__ nb_k, const int *__restrict__ no_k, int nk, double inv_nk,
                              double q0b, int q0_on, double2 *const *__restrict__ kp) {
    int ik = blockIdx.y;
    int nb = nb_k[ik], no = no_k[ik];
    const double2 *A = vacc[ik];
    const double2 *K = kp ? kp[ik] : nullptr;
    double2 *V = Vout[ik];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nb * nb; e += gridDim.x * blockDim.x) {
        int n = e / nb, n2 = e % nb;
        double2 a = A[e];
        double2 v = make_double2(-inv_nk * a.x, -inv_nk * a.y);
        if (q0_on && n == n2 && n < no) v.x -= q0b;
        if (K) { v.x += K[e].x; v.y += K[e].y; }
        V[e] = v;
    }
}

// D[a][m][n] = <phi_m | d/dq_a Phi_n> = -i p[a][m][n] / (eps[n] - eps[m]), zero for
// m = n and for degenerate pairs (first-order k.p, Appendix A).
__device__ __forceinline__ double2 kp_d(const double2 *p, const double *eps, int nb, int a, int m, int n, double tol) {
    const double de = eps[n] - eps[m];
    if (m == n || fabs(de) < tol) return make_double2(0.0, 0.0);
    const double2 x = p[((size_t)a * nb + m) * nb + n];
    return make_double2(x.y / de, -x.x / de);
}

// One thread per (k, n1, n2): the spherical average Abar of the second-order
// terms of the integrand at q = 0 and the term -Abar / (N_k Omega) it adds to V^x.
__global__ void kp_term_kernel(const double *const *__restrict__ eps_k, const double2 *const *__restrict__ p_k,
                               double2 *const *__restrict__ kp_k, const int *__restrict__ nb_k,
                               const int *__restrict__ no_k, double nk_omega, double tol) {
    const int ik = blockIdx.y;
    const int nb = nb_k[ik], no = no_k[ik];
    const double *eps = eps_k[ik];
    const double2 *p = p_k[ik];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nb * nb; e += gridDim.x * blockDim.x) {
        const int n1 = e / nb, n2 = e % nb;
        double2 acc = make_double2(0.0, 0.0);
        for (int a = 0; a < 3; ++a) {
            for (int n = 0; n < no; ++n)
                acc = cfma_conj(kp_d(p, eps, nb, a, n2, n, tol), kp_d(p, eps, nb, a, n1, n, tol), acc);
            if (n1 < no && n2 < no)
                for (int m = 0; m < nb; ++m) {
                    const double2 t = cfma_conj(kp_d(p, eps, nb, a, m, n1, tol), kp_d(p, eps, nb, a, m, n2, tol),
                                                make_double2(0.0, 0.0));
                    acc.x -= t.x;
                    acc.y -= t.y;
                }
        }
        const double f = -(4.0 * 3.14159265358979323846 / 3.0) / nk_omega;
        kp_k[ik][e] = make_double2(f * acc.x, f * acc.y);
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
                         int real_part, double2 *const *d_vacc, const int *d_nb_k, int nb_max, cudaStream_t st) {
    if (nk_in_batch == 0) return;
    int nx = (nb_max * nb_max + 255) / 256;
    if (nx > 64) nx = 64;
    dim3 grid((unsigned)nx, (unsigned)nk_in_batch);
    reduce_pairs_kernel<<<grid, 256, 0, st>>>(d_pairs, d_kstart, d_klist_pairs, d_klist, d_praw, d_praw_off, NB,
                                              raw_format, real_part, d_vacc, d_nb_k);
}

void launch_finish(double2 *const *d_vacc, double2 *const *d_V, const int *d_nb_k, const int *d_no_k, int nk,
                   int nb_max, double inv_nk, double q0b, int q0_on, double2 *const *d_kp, double *d_Ex,
                   cudaStream_t st) {
    int nx = (nb_max * nb_max + 255) / 256;
    if (nx > 64) nx = 64;
    dim3 grid((unsigned)nx, (unsigned)nk);
    finish_kernel<<<grid, 256, 0, st>>>(d_vacc, d_V, d_nb_k, d_no_k, nk, inv_nk, q0b, q0_on, d_kp);
    energy_kernel<<<1, 256, 0, st>>>(d_V, d_nb_k, d_no_k, nk, inv_nk, d_Ex);
}

void launch_kp_term(const double *const *d_eps, const double2 *const *d_p, double2 *const *d_kp, const int *d_nb_k,
                    const int *d_no_k, int nk, int nb_max, double nk_omega, double deg_tol, cudaStream_t st) {
    int nx = (nb_max * nb_max + 127) / 128;
    if (nx > 1024) nx = 1024;
    dim3 grid((unsigned)nx, (unsigned)nk);
    kp_term_kernel<<<grid, 128, 0, st>>>(d_eps, d_p, d_kp, d_nb_k, d_no_k, nk_omega, deg_tol);
}

}  // namespace hfx
