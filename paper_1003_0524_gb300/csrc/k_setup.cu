// k_setup.cu -- once-per-context and once-per-SCF-cycle kernels, all FP64:
// Gaunt table, multipole transforms, step function, Coulomb-matrix transform,
// split embedding of the transformed Coulomb matrix, q->0 bracket.
#include <cmath>

#include "hfx_internal.cuh"
#include "tc_ptx.cuh"

namespace hfx {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kGL = 24;  // Gauss-Legendre nodes: exact for polynomial degree <= 47

// Normalised associated Legendre functions (Condon-Shortley phase included):
// Y_lm(theta, phi) = Pbar_lm(cos theta) e^{i m phi} for m >= 0.
__device__ void pbar_all(double x, int lmax, double *out /* [(lmax+1)^2] by l*l+l+m, m>=0 used */) {
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 1.0 / sqrt(4.0 * kPi);
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) pmm = -sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm;
        out[m * m + m + m] = pmm;
        if (m + 1 <= lmax) {
            double p1 = sqrt(2.0 * m + 3.0) * x * pmm;
            out[(m + 1) * (m + 1) + (m + 1) + m] = p1;
            double pl2 = pmm, pl1 = p1;
            for (int l = m + 2; l <= lmax; ++l) {
                double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                double b = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
                double pl = a * (x * pl1 - b * pl2);
                out[l * l + l + m] = pl;
                pl2 = pl1;
                pl1 = pl;
            }
        }
    }
}

__device__ double pbar_signed(const double *tab, int l, int m) {
    // Y_{l,-m} = (-1)^m conj(Y_{lm}) => Pbar_{l,-m} = (-1)^m Pbar_{lm}
    if (m >= 0) return tab[l * l + l + m];
    double v = tab[l * l + l - m];
    return (m & 1) ? -v : v;
}

__global__ void gaunt_kernel(double *out, int Lmax, int lmax) {
    __shared__ double xs[kGL], ws[kGL];
    if (threadIdx.x < kGL) {
        int i = threadIdx.x;
        double x = cos(kPi * (i + 0.75) / (kGL + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int j = 1; j < kGL; ++j) {
                double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = kGL * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        xs[i] = x;
        ws[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    __syncthreads();
    int nLM = (Lmax + 1) * (Lmax + 1), nlm = (lmax + 1) * (lmax + 1);
    int total = nLM * nlm * (lmax + 1);
    int lm_all = (max(Lmax, lmax) + 1) * (max(Lmax, lmax) + 1);
    double tab[(kMaxL + 1) * (kMaxL + 1)];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int l2 = e % (lmax + 1);
        int lm = (e / (lmax + 1)) % nlm;
        int LM = e / ((lmax + 1) * nlm);
        int L = (int)floor(sqrt((double)LM) + 1e-9), M = LM - L * L - L;
        int l = (int)floor(sqrt((double)lm) + 1e-9), m = lm - l * l - l;
        int m2 = m + M;
        double val = 0.0;
        bool tri = (l2 >= abs(L - l)) && (l2 <= L + l) && (((L + l + l2) & 1) == 0);
        if (abs(m2) <= l2 && tri) {
            double acc = 0.0;
            for (int i = 0; i < kGL; ++i) {
                pbar_all(xs[i], max(max(Lmax, lmax), 0), tab);
                acc += ws[i] * pbar_signed(tab, L, M) * pbar_signed(tab, l, m) * pbar_signed(tab, l2, m2);
            }
            // int Y*_LM Y*_lm Y_l2m2 dphi = 2 pi (m2 = M + m)
            val = 2.0 * kPi * acc;
        }
        (void)lm_all;
        out[e] = val;
    }
}

// Orthogonal T_{aL}: first row mu/|mu| (the only function that keeps a
// multipole moment), remaining rows a Gram-Schmidt completion from the unit
// vectors (Sec. III.C; any orthonormal completion gives the same V^x).
__global__ void transform_T_kernel(const double *mu, double *T, int n_atoms, int Lmax, int P) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_atoms * (Lmax + 1)) return;
    const double *m = mu + (size_t)idx * P;
    double *t = T + (size_t)idx * P * P;
    double nrm = 0.0;
    for (int i = 0; i < P; ++i) nrm += m[i] * m[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < P * P; ++i) t[i] = 0.0;
    if (nrm == 0.0) {
        for (int i = 0; i < P; ++i) t[i * P + i] = 1.0;
        return;
    }
    for (int j = 0; j < P; ++j) t[j] = m[j] / nrm;
    int row = 1;
    for (int e = 0; e < P && row < P; ++e) {
        double w[kMaxP];
        for (int j = 0; j < P; ++j) w[j] = (j == e) ? 1.0 : 0.0;
        for (int pass = 0; pass < 2; ++pass)
            for (int r = 0; r < row; ++r) {
                double d = 0.0;
                for (int j = 0; j < P; ++j) d += t[r * P + j] * w[j];
                for (int j = 0; j < P; ++j) w[j] -= d * t[r * P + j];
            }
        double wn = 0.0;
        for (int j = 0; j < P; ++j) wn += w[j] * w[j];
        wn = sqrt(wn);
        if (wn < 1e-8) continue;
        for (int j = 0; j < P; ++j) t[row * P + j] = w[j] / wn;
        ++row;
    }
}

// Theta_K = delta_K0 - (1/Omega) sum_a e^{-i K.R_a} 4 pi S_a^3 j1(|K| S_a)/(|K| S_a)
// (Fourier coefficients of the interstitial step function, Eq. step function).
__global__ void theta_kernel(double2 *out, int lo0, int lo1, int lo2, int d0, int d1, int d2, double b00,
                             double b01, double b02, double b10, double b11, double b12, double b20, double b21,
                             double b22, double omega, const double *posf, const double *rmt, int n_atoms) {
    long long total = (long long)d0 * d1 * d2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int z = (int)(e % d2), y = (int)((e / d2) % d1), x = (int)(e / ((long long)d1 * d2));
        int K0 = lo0 + x, K1 = lo1 + y, K2 = lo2 + z;
        double kx = K0 * b00 + K1 * b10 + K2 * b20;
        double ky = K0 * b01 + K1 * b11 + K2 * b21;
        double kz = K0 * b02 + K1 * b12 + K2 * b22;
        double kn = sqrt(kx * kx + ky * ky + kz * kz);
        bool zero = (K0 == 0 && K1 == 0 && K2 == 0);
        double re = zero ? 1.0 : 0.0, im = 0.0;
        for (int a = 0; a < n_atoms; ++a) {
            double S = rmt[a];
            double x1 = kn * S;
            double f;
            if (zero) {
                f = 4.0 * kPi * S * S * S / 3.0;
            } else if (x1 < 1e-3) {
                f = 4.0 * kPi * S * S * S * (1.0 / 3.0 - x1 * x1 / 30.0);
            } else {
                double sx, cx;
                sincos(x1, &sx, &cx);
                f = 4.0 * kPi * S * S * S * (sx / (x1 * x1) - cx / x1) / x1;
            }
            double ph = 2.0 * kPi * (K0 * posf[3 * a] + K1 * posf[3 * a + 1] + K2 * posf[3 * a + 2]);
            double sp, cp;
            sincos(ph, &sp, &cp);
            re -= f * cp / omega;
            im += f * sp / omega;
        }
        out[e] = make_double2(re, im);
    }
}

// Classify a permuted MPB index (sparse layout):
// kind 0: mu=0 function (channel ch, transformed index i >= 1)
// kind 1: mu!=0 function of channel ch (i = 0)
// kind 2: interstitial plane wave g
struct PIdx { int kind, ch, i, g; };

__device__ __forceinline__ PIdx classify(int p, int N0, int nch, int P) {
    PIdx r;
    if (p < N0) { r.kind = 0; r.ch = p / (P - 1); r.i = 1 + p % (P - 1); r.g = -1; }
    else if (p < N0 + nch) { r.kind = 1; r.ch = p - N0; r.i = 0; r.g = -1; }
    else { r.kind = 2; r.ch = -1; r.i = -1; r.g = p - N0 - nch; }
    return r;
}

// v_t[p][q] = sum_{s,s'} T_p[s] v[orig(p,s)][orig(q,s')] T_q[s'] in the permuted
// order [mu=0 | mu!=0 | IPW] (sparse) or the original order without transform.
__global__ void transform_v_kernel(const double2 *v, double2 *VD, double2 *VB, const double *T, int n_atoms,
                                   int Lmax, int P, int nipw, int sparse, unsigned long long *offmax,
                                   unsigned long long *absmax) {
    int nLM = (Lmax + 1) * (Lmax + 1);
    int nch = n_atoms * nLM, nmt = nch * P, naux = nmt + nipw;
    int N0 = sparse ? nch * (P - 1) : 0;
    long long total = (long long)naux * naux;
    // running maxima of |v_t| and of the elements off the pattern, per thread
    // (non-negative doubles order like their bit patterns), one atomic per warp
    unsigned long long tabs = 0, toff = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int p = (int)(e / naux), q = (int)(e % naux);
        if (!sparse) {
            double2 val = v[e];
            VD[e] = val;
            tabs = max(tabs, (unsigned long long)__double_as_longlong(fabs(val.x) + fabs(val.y)));
            continue;
        }
        PIdx a = classify(p, N0, nch, P), b = classify(q, N0, nch, P);
        double2 acc = make_double2(0.0, 0.0);
        if (a.kind == 2 && b.kind == 2) {
            acc = v[(size_t)(nmt + a.g) * naux + nmt + b.g];
        } else if (a.kind == 2) {
            const double *Tb = T + ((size_t)(b.ch / nLM) * (Lmax + 1) + (int)floor(sqrt((double)(b.ch % nLM)) + 1e-9)) * P * P + b.i * P;
            for (int s2 = 0; s2 < P; ++s2) {
                double2 x = v[(size_t)(nmt + a.g) * naux + b.ch * P + s2];
                acc.x += Tb[s2] * x.x;
                acc.y += Tb[s2] * x.y;
            }
        } else if (b.kind == 2) {
            const double *Ta = T + ((size_t)(a.ch / nLM) * (Lmax + 1) + (int)floor(sqrt((double)(a.ch % nLM)) + 1e-9)) * P * P + a.i * P;
            for (int s1 = 0; s1 < P; ++s1) {
                double2 x = v[(size_t)(a.ch * P + s1) * naux + nmt + b.g];
                acc.x += Ta[s1] * x.x;
                acc.y += Ta[s1] * x.y;
            }
        } else {
            const double *Ta = T + ((size_t)(a.ch / nLM) * (Lmax + 1) + (int)floor(sqrt((double)(a.ch % nLM)) + 1e-9)) * P * P + a.i * P;
            const double *Tb = T + ((size_t)(b.ch / nLM) * (Lmax + 1) + (int)floor(sqrt((double)(b.ch % nLM)) + 1e-9)) * P * P + b.i * P;
            for (int s1 = 0; s1 < P; ++s1) {
                double2 row = make_double2(0.0, 0.0);
                for (int s2 = 0; s2 < P; ++s2) {
                    double2 x = v[(size_t)(a.ch * P + s1) * naux + b.ch * P + s2];
                    row.x += Tb[s2] * x.x;
                    row.y += Tb[s2] * x.y;
                }
                acc.x += Ta[s1] * row.x;
                acc.y += Ta[s1] * row.y;
            }
        }
        double mag = fabs(acc.x) + fabs(acc.y);
        tabs = max(tabs, (unsigned long long)__double_as_longlong(mag));
        // pattern of Fig. 1: a mu=0 function couples only inside its own channel
        bool allowed = true;
        if (a.kind == 0 && b.ch != a.ch) allowed = false;
        if (b.kind == 0 && a.ch != b.ch) allowed = false;
        if (!allowed) {
            toff = max(toff, (unsigned long long)__double_as_longlong(mag));
            acc = make_double2(0.0, 0.0);
        }
        if (p >= N0) {
            VD[(size_t)(p - N0) * naux + q] = acc;
        } else if (allowed) {
            int slot = (b.kind == 1) ? 0 : b.i;  // 0: the channel's mu!=0 function
            VB[((size_t)a.ch * (P - 1) + (a.i - 1)) * P + slot] = acc;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tabs = max(tabs, __shfl_xor_sync(0xffffffffu, tabs, o));
        toff = max(toff, __shfl_xor_sync(0xffffffffu, toff, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (tabs) atomicMax(absmax, tabs);
        if (toff) atomicMax(offmax, toff);
    }
}

// Element (r, c) of the real embedding [[Ur, -Ui], [Ui, Ur]] of the
// dense-block rows of U, the upper triangle of v_t with half its diagonal
// (v_t = U + U^H for Hermitian v_t, so Z^H v_t Z = P' + P'^H with P' = Z^H U Z):
// rows [Re D (Dpad) | Im D (Dpad)], columns [Re (N0pad + Dpad) | Im (N0pad +
// Dpad)] (zero in the padding).  In the order [mu=0 | dense], the mu = 0
// columns of the dense-block rows lie below the diagonal and are zero in U.
__device__ __forceinline__ double ap_elem(const double2 *VD, int r, int c, int D, int naux, int N0, int N0pad,
                                         int Dpad, int interleave) {
    int HS = N0pad + Dpad;
    // interleaved: row 2r real, 2r + 1 imaginary part of row r; else real rows
    // [0, D), imaginary rows [D, 2D)
    int rim = interleave ? (r & 1) : (r >= D), rr = interleave ? (r >> 1) : (rim ? r - D : r);
    int cim = c >= HS, u = cim ? c - HS : c;
    if (rr >= D || u < N0pad) return 0.0;
    const int d = u - N0pad;                  // dense column index
    if (d >= naux - N0 || d < rr) return 0.0;
    double2 val = VD[(size_t)rr * naux + N0 + d];
    if (d == rr) { val.x *= 0.5; val.y *= 0.5; }
    if (!rim && !cim) return val.x;
    if (!rim && cim) return -val.y;
    if (rim && !cim) return val.y;
    return val.x;
}

// Fixed-point slices of A' (one block per row; rows 2r and 2r + 1 the real and
// imaginary parts of row r, or with a real v_t rows [0, D) real and [D, 2D)
// imaginary; the rest of the 2 Dpad rows zero): exponent e_r with
// max_c |A'_rc| < 2^e_r, then the four slices of tc_ptx.cuh per element, stored
// as BF16 planes [4][2 Dpad][RS] (the slice format of k_contract_tc.cu).
__global__ void build_ap_kernel(const double2 *VD, __nv_bfloat16 *Ap, int *aexp, int D, int naux, int N0, int N0pad,
                                int Dpad, int RS, int interleave) {
    int r = blockIdx.x;
    long long plane = 2LL * Dpad * RS;
    __shared__ unsigned long long red[256];
    unsigned long long mx = 0;
    for (int c = threadIdx.x; c < RS; c += blockDim.x)
        mx = max(mx, tc::abs_bits(ap_elem(VD, r, c, D, naux, N0, N0pad, Dpad, interleave)));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    const int e = tc::line_exp_bits(red[0]);
    if (threadIdx.x == 0) aexp[r] = e;
    for (int c = threadIdx.x; c < RS; c += blockDim.x) {
        __nv_bfloat16 sl[tc::NPL];
        tc::slice4(ap_elem(VD, r, c, D, naux, N0, N0pad, Dpad, interleave), e, sl);
        for (int i = 0; i < tc::NPL; ++i) Ap[i * plane + (long long)r * RS + c] = sl[i];
    }
}

// Partial sums of e^{-beta|q+G|^2}/|q+G|^2 over 0 < |q+G| <= q0: one block
// per (q, G_x) slab, deterministic block reduction.
__global__ void q0_partial_kernel(double *partial, int m0, int m1, int m2, double b00, double b01, double b02,
                                  double b10, double b11, double b12, double b20, double b21, double b22,
                                  double beta, double q0, int bx, int by, int bz) {
    int slab = blockIdx.x;
    int nx = 2 * bx + 1;
    int iq = slab / nx, gx = slab % nx - bx;
    int j2 = iq % m2, j1 = (iq / m2) % m1, j0 = iq / (m1 * m2);
    double f0 = (double)j0 / m0 + gx;
    double acc = 0.0;
    int ny = 2 * by + 1, nz = 2 * bz + 1;
    for (int t = threadIdx.x; t < ny * nz; t += blockDim.x) {
        double f1 = (double)j1 / m1 + (t / nz - by);
        double f2 = (double)j2 / m2 + (t % nz - bz);
        double cx = f0 * b00 + f1 * b10 + f2 * b20;
        double cy = f0 * b01 + f1 * b11 + f2 * b21;
        double cz = f0 * b02 + f1 * b12 + f2 * b22;
        double q2 = cx * cx + cy * cy + cz * cz;
        if (q2 > 0.0 && q2 <= q0 * q0) acc += exp(-beta * q2) / q2;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[slab] = red[0];
}

__global__ void q0_final_kernel(const double *partial, int n, double *out, double beta, double q0, double nk,
                                double omega) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double integral = erf(sqrt(beta) * q0) / sqrt(kPi * beta);
        out[0] = integral - 4.0 * kPi / (nk * omega) * red[0];
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 32) g = 152LL * 32;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

void launch_gaunt(double *d_gaunt, int Lmax, int lmax, cudaStream_t st) {
    int total = (Lmax + 1) * (Lmax + 1) * (lmax + 1) * (lmax + 1) * (lmax + 1);
    gaunt_kernel<<<grid_for(total, 128), 128, 0, st>>>(d_gaunt, Lmax, lmax);
}

void launch_transform_T(const double *d_mu, double *d_T, int n_atoms, int Lmax, int P, cudaStream_t st) {
    int n = n_atoms * (Lmax + 1);
    transform_T_kernel<<<(n + 63) / 64, 64, 0, st>>>(d_mu, d_T, n_atoms, Lmax, P);
}

void launch_theta(double2 *d_theta, const int lo[3], const int dim[3], const double *B, double omega,
                  const double *d_posf, const double *d_rmt, int n_atoms, cudaStream_t st) {
    long long n = (long long)dim[0] * dim[1] * dim[2];
    theta_kernel<<<grid_for(n, 256), 256, 0, st>>>(d_theta, lo[0], lo[1], lo[2], dim[0], dim[1], dim[2], B[0],
                                                   B[1], B[2], B[3], B[4], B[5], B[6], B[7], B[8], omega,
                                                   d_posf, d_rmt, n_atoms);
}

void launch_transform_v(const double2 *d_v, double2 *d_VD, double2 *d_VB, const double *d_T, int n_atoms,
                        int Lmax, int P, int nipw, int sparse, unsigned long long *d_offmax,
                        unsigned long long *d_absmax, cudaStream_t st) {
    long long naux = (long long)n_atoms * (Lmax + 1) * (Lmax + 1) * P + nipw;
    transform_v_kernel<<<grid_for(naux * naux, 256), 256, 0, st>>>(d_v, d_VD, d_VB, d_T, n_atoms, Lmax, P, nipw,
                                                                  sparse, d_offmax, d_absmax);
}

void launch_build_ap(const double2 *d_VD, __nv_bfloat16 *d_Ap, int *d_aexp, int D, int naux, int N0, int N0pad,
                     int Dpad, int RS, int interleave, cudaStream_t st) {
    build_ap_kernel<<<2 * Dpad, 256, 0, st>>>(d_VD, d_Ap, d_aexp, D, naux, N0, N0pad, Dpad, RS, interleave);
}

// q->0 bracket with box bounds from the lattice (|n_i| <= q0 |a_i| / 2pi + 2).
void launch_q0_bracket_impl(double *d_out, double *d_partial, const int mesh[3], const double *B, double omega,
                            double beta, const double *lattice, cudaStream_t st) {
    double q0 = sqrt(-log(beta) / beta);
    int bnd[3];
    for (int i = 0; i < 3; ++i) {
        double an = sqrt(lattice[3 * i] * lattice[3 * i] + lattice[3 * i + 1] * lattice[3 * i + 1] +
                         lattice[3 * i + 2] * lattice[3 * i + 2]);
        bnd[i] = (int)ceil(q0 * an / (2.0 * kPi)) + 2;
    }
    int nk = mesh[0] * mesh[1] * mesh[2];
    int nslab = nk * (2 * bnd[0] + 1);
    q0_partial_kernel<<<nslab, 256, 0, st>>>(d_partial, mesh[0], mesh[1], mesh[2], B[0], B[1], B[2], B[3], B[4],
                                             B[5], B[6], B[7], B[8], beta, q0, bnd[0], bnd[1], bnd[2]);
    q0_final_kernel<<<1, 256, 0, st>>>(d_partial, nslab, d_out, beta, q0, (double)nk, omega);
}

size_t q0_partial_count(const int mesh[3], double beta, const double *lattice) {
    double q0 = sqrt(-log(beta) / beta);
    double an = sqrt(lattice[0] * lattice[0] + lattice[1] * lattice[1] + lattice[2] * lattice[2]);
    int b0 = (int)ceil(q0 * an / (2.0 * kPi)) + 2;
    return (size_t)mesh[0] * mesh[1] * mesh[2] * (2 * b0 + 1);
}

}  // namespace hfx

// =====================================================================
// Allocation-free variant of the q->0 bracket.
//
// Some callers cannot allocate device memory at the point where they need
// this number: processes whose device memory is entirely owned by another
// allocator (for example a framework's caching pool that has reserved the
// device), and code paths that must not trigger the implicit device-wide
// synchronisation that cudaMalloc/cudaFree may perform.  For them the
// per-slab partial sums of the reduction live in the fixed array below
// instead of a cudaMalloc'd buffer.  The array is a file-scope device
// variable: every GPU that loads this library holds it (512 KiB) until the
// process exits, and every call shares it.
// =====================================================================
namespace hfx {
namespace {

constexpr int kQ0ScratchMax = 65536;   // partial sums (doubles) the array holds
static __device__ __align__(256) double g_q0_scratch[kQ0ScratchMax];

// In host code the name g_q0_scratch is only a host-side stand-in, never a
// device address: every call resolves the current device's address with
// cudaGetSymbolAddress (which allocates nothing), so no cached pointer is
// shared between host threads or outlives a device reset.

__global__ void q0_final_to_kernel(const double *partial, int n, double *out, double beta, double q0, double nk,
                                   double omega) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = erf(sqrt(beta) * q0) / sqrt(kPi * beta) - 4.0 * kPi / (nk * omega) * red[0];
}

}  // namespace

}  // namespace hfx

extern "C" int hfx_q0_bracket_noalloc(const double *lattice, const int *mesh, double beta, double *bracket_dev,
                                      void *stream) {
    using namespace hfx;
    if (!lattice || !mesh || !bracket_dev || !(beta > 0.0 && beta < 1.0)) return HFX_EINVAL;
    for (int i = 0; i < 3; ++i)
        if (mesh[i] < 1 || mesh[i] > 64) return HFX_EINVAL;
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(lattice[i])) return HFX_ENONFINITE;
    const double *a = lattice;
    double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
    if (!(fabs(det) > 1e-9)) return HFX_EINVAL;
    // reciprocal rows b_i = 2 pi (A^{-1})^T, evaluated as in hfx_create
    double inv[9], B[9];
    inv[0] = (a[4] * a[8] - a[5] * a[7]) / det; inv[1] = (a[2] * a[7] - a[1] * a[8]) / det; inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
    inv[3] = (a[5] * a[6] - a[3] * a[8]) / det; inv[4] = (a[0] * a[8] - a[2] * a[6]) / det; inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
    inv[6] = (a[3] * a[7] - a[4] * a[6]) / det; inv[7] = (a[1] * a[6] - a[0] * a[7]) / det; inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[3 * i + j] = 2.0 * M_PI * inv[3 * j + i];
    size_t nslab = q0_partial_count(mesh, beta, lattice);
    if (nslab > (size_t)kQ0ScratchMax) return HFX_EUNSUPPORTED;   // k mesh x G box too large for the fixed array
    // the array's address on the current device (the first call on a device
    // also loads the library's module there)
    double *partial = nullptr;
    if (cudaGetSymbolAddress((void **)&partial, g_q0_scratch) != cudaSuccess || !partial) {
        cudaGetLastError();
        return HFX_EDEVICE;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double q0 = sqrt(-log(beta) / beta);
    int bnd[3];
    for (int i = 0; i < 3; ++i) {
        double an = sqrt(lattice[3 * i] * lattice[3 * i] + lattice[3 * i + 1] * lattice[3 * i + 1] +
                         lattice[3 * i + 2] * lattice[3 * i + 2]);
        bnd[i] = (int)ceil(q0 * an / (2.0 * kPi)) + 2;
    }
    int nk = mesh[0] * mesh[1] * mesh[2];
    // every partial sum [0, nslab) is written before it is read: nothing to clear
    q0_partial_kernel<<<(unsigned)nslab, 256, 0, st>>>(partial, mesh[0], mesh[1], mesh[2], B[0], B[1], B[2], B[3], B[4],
                                                       B[5], B[6], B[7], B[8], beta, q0, bnd[0], bnd[1], bnd[2]);
    q0_final_to_kernel<<<1, 256, 0, st>>>(partial, (int)nslab, bracket_dev, beta, q0, (double)nk, fabs(det));
    return cudaGetLastError() == cudaSuccess ? HFX_OK : HFX_EDEVICE;
}
