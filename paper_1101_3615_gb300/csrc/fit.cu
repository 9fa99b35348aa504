// Randomized fit of the inverse-Hessian symbol expansion and its application
// as a preconditioner (sm_103a, FP64).
//
// probe_fit (Sec. 1.4): with x_j = H y_j, the columns of the least-squares
// problem are (B_i x_j)(x) = alpha_lam(x) * IFFT[beta_m(k) FFT(x_j)](x),
// i = (lam, m), m = (angular a, radial q).  One batched D2Z transform of the
// p zero-padded trials, one multiply + batched Z2D transform per distinct k
// multiplier beta_m; then the least-squares problem min ||A c - y|| over the
// rows of all trials is solved through a QR factorisation of A in FP64 by
// CholeskyQR2 (Cholesky QR with one reorthogonalisation):
//     pass 1:  A^T A = R1^T R1                       (Cholesky)
//     pass 2:  Q1 = A R1^{-1} row by row, Q1^T Q1 = R2^T R2, z = Q1^T y
//     A = Q R with Q = Q1 R2^{-1}, R = R2 R1:  c = R^{-1} Q^T y = R1^{-1} R2^{-1} R2^{-T} z.
// The Gram matrix of the reorthogonalised Q1 is within a few units of round-off
// of the identity whenever cond(A) is below about 1e7, so the solution has the
// accuracy of a Householder QR (error ~ cond(A) eps) instead of the
// cond(A)^2 eps of the normal equations M c = A^T y that Sec. 1.4 writes; the
// first Cholesky factorisation fails (PROBE_ERR_STATE) only when A is
// numerically rank deficient.  Gram matrices: P <= 64 -- columns formed on the
// fly in shared memory, 32 rows at a time (pass 2 applies R1^{-1} to the staged
// rows in shared memory); P up to 1024 -- [A | y] formed in column-major chunks
// of about 256 MB, R1^{-1} applied row by row, and a tiled FP64 Gram kernel.
// A second pass forms ||y - sum_i c_i B_i x|| / ||y||.
//
// probe_apply_precond (end of Sec. 1.5): one D2Z transform of the image, one
// combined multiplier gamma_lam(k) = sum_m c_(lam,m) beta_m(k) per spatial mode,
// a batched Z2D transform, and out = sum_lam alpha_lam * w_lam.
//
// cuFFT provides the plain FFTs; every other step is a kernel of this file.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "common.cuh"
#include "handle.h"
#include "internal.h"

namespace probe {

constexpr int kMaxTerms = 1024;   // P = nspatial x nangular x nradial
constexpr int kMaxSmall = 64;     // P <= 64: Gram pairs accumulated in one CTA's registers
constexpr int kMaxSpatial = 32;
constexpr int kMaxAngular = 16;
constexpr int kMaxRadial = 16;
constexpr int kMaxMult = 32;      // nangular * nradial
constexpr int kGramRows = 32;     // rows staged per Gram iteration
constexpr int kGramBlocks = 608;  // 4 CTAs per SM
constexpr long long kChunkBytes = 256ll << 20;  // large-P path: [A | y] chunk size

struct BasisDev {
    int ndim;
    int n[3];          // interior sizes (z, y, x); 2D uses n[1] = 1
    int Nf[3];         // FFT sizes
    int fp;            // fft pad (y axis unpadded in 2D)
    double h[3];
    int nspatial, nangular, nradial, NM, P;
    int spatial[kMaxSpatial][3];
    int angular[kMaxAngular];
    double L, order;
    long long Nreal, Ncplx, npts;
};

struct FitCache {
    std::map<std::tuple<int, int, int, int, int>, cufftHandle> plans;  // (ndim, Nz, Ny, Nx, kind*batch)
    DevBuf xr, Xc, Wc, w, beta, alpha, part, coef, misc;
    DevBuf gram, L1, L2, chunk;  // CholeskyQR2: Gram matrix, the two Cholesky factors, [A | y] chunk
};

void fit_cache_destroy(probe_t h) {
    if (!h || !h->fit) return;
    for (auto& kv : h->fit->plans) cufftDestroy(kv.second);
    DevBuf* bufs[] = {&h->fit->xr, &h->fit->Xc, &h->fit->Wc, &h->fit->w,  &h->fit->beta, &h->fit->alpha,
                      &h->fit->part, &h->fit->coef, &h->fit->misc, &h->fit->gram, &h->fit->L1, &h->fit->L2,
                      &h->fit->chunk};
    for (DevBuf* b : bufs)
        if (b->p) cudaFree(b->p);
    delete h->fit;
    h->fit = nullptr;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void unravel(long long i, const BasisDev& B, int& iz, int& iy, int& ix) {
    ix = (int)(i % B.n[2]);
    const long long r = i / B.n[2];
    iy = (int)(r % B.n[1]);
    iz = (int)(r / B.n[1]);
}

__device__ __forceinline__ long long fft_index(const BasisDev& B, int iz, int iy, int ix) {
    const int fpy = (B.ndim == 3) ? B.fp : 0;
    return ((long long)(iz + B.fp) * B.Nf[1] + (iy + fpy)) * B.Nf[2] + (ix + B.fp);
}

// zero-padded FP64 copies of `cnt` interior FP32 fields
__global__ void k_fit_pad(const float* __restrict__ src, double* __restrict__ dst, int cnt, BasisDev B) {
    const long long tot = (long long)cnt * B.npts;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / B.npts);
        int iz, iy, ix;
        unravel(i - (long long)j * B.npts, B, iz, iy, ix);
        dst[(long long)j * B.Nreal + fft_index(B, iz, iy, ix)] = (double)src[i];
    }
}

// beta_m(k) for every multiplier m = a * nradial + q on the half (real-FFT) grid
__global__ void k_fit_beta(double* __restrict__ beta, BasisDev B) {
    const long long tot = (long long)B.NM * B.Ncplx;
    const int hx = B.Nf[2] / 2 + 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(i / B.Ncplx);
        long long r = i - (long long)m * B.Ncplx;
        const int jx = (int)(r % hx);
        r /= hx;
        const int jy = (int)(r % B.Nf[1]);
        const int jz = (int)(r / B.Nf[1]);
        const int a = m / B.nradial, q = m % B.nradial;
        auto freq = [](int j, int N) { return (j <= (N - 1) / 2) ? j : j - N; };
        const double two_pi = 6.283185307179586476925286766559;
        const double kz = two_pi * freq(jz, B.Nf[0]) / (B.Nf[0] * B.h[0]);
        const double ky = (B.ndim == 3) ? two_pi * freq(jy, B.Nf[1]) / (B.Nf[1] * B.h[1]) : 0.0;
        const double kx = two_pi * jx / (B.Nf[2] * B.h[2]);
        bool nyq = ((B.Nf[0] % 2) == 0 && jz == B.Nf[0] / 2) || ((B.Nf[2] % 2) == 0 && jx == B.Nf[2] / 2);
        if (B.ndim == 3) nyq = nyq || ((B.Nf[1] % 2) == 0 && jy == B.Nf[1] / 2);
        const double kn = sqrt(kz * kz + ky * ky + kx * kx);
        double v = 0.0;
        if (kn > 0.0 && !nyq) {
            double A;
            const int ang = B.angular[a];
            if (B.ndim == 2) {
                const double th = atan2(kz, kx);
                A = (ang == 0) ? 1.0 : (ang > 0 ? cos(ang * th) : sin(-ang * th));
            } else {
                const double uz = kz / kn, uy = ky / kn, ux = kx / kn;
                switch (ang) {
                    case 0: A = 1.0; break;
                    case 1: A = ux * uy; break;
                    case 2: A = uy * uz; break;
                    case 3: A = ux * uz; break;
                    case 4: A = ux * ux - uy * uy; break;
                    default: A = 3.0 * uz * uz - 1.0; break;
                }
            }
            double t = (kn - B.L) / (kn + B.L);
            t = fmin(1.0, fmax(-1.0, t));
            v = A * cos(q * acos(t)) * pow(kn, B.order);
        }
        beta[i] = v;
    }
}

// alpha tables: alpha[lam][axis][i] (axis order z, y, x; unused axes hold 1)
__global__ void k_fit_alpha(double* __restrict__ alpha, BasisDev B, int nmax) {
    const long long tot = (long long)B.nspatial * 3 * nmax;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int lam = (int)(i / (3 * nmax));
        const int rem = (int)(i - (long long)lam * 3 * nmax);
        const int ax = rem / nmax, idx = rem % nmax;
        const int n = B.n[ax];
        const int k = (B.ndim == 2) ? (ax == 0 ? B.spatial[lam][0] : (ax == 2 ? B.spatial[lam][1] : 0))
                                    : B.spatial[lam][ax];
        const double two_pi = 6.283185307179586476925286766559;
        double v = 1.0;
        if (idx < n && k != 0)
            v = (k > 0) ? cos(two_pi * k * idx / n) : sin(two_pi * (-k) * idx / n);
        alpha[i] = v;
    }
}

// out[c][j][k] = mult[c or 0][k] * X[j][k] / N  for the spectra of cnt fields
__global__ void k_fit_mult(const double2* __restrict__ X, const double* __restrict__ mult, double2* __restrict__ out,
                           int nmult, int cnt, long long Ncplx, double invN) {
    const long long tot = (long long)nmult * cnt * Ncplx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i % Ncplx;
        const long long mj = i / Ncplx;
        const int j = (int)(mj % cnt);
        const int m = (int)(mj / cnt);
        const double b = mult[(long long)m * Ncplx + k] * invN;
        const double2 x = X[(long long)j * Ncplx + k];
        out[i] = make_double2(b * x.x, b * x.y);
    }
}

// gamma_lam(k) = sum_m c[lam*NM + m] beta_m(k)
__global__ void k_precond_gamma(const double* __restrict__ beta, const double* __restrict__ c,
                                double* __restrict__ gamma, BasisDev B) {
    const long long tot = (long long)B.nspatial * B.Ncplx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int lam = (int)(i / B.Ncplx);
        const long long k = i - (long long)lam * B.Ncplx;
        double g = 0.0;
        for (int m = 0; m < B.NM; ++m) g += c[lam * B.NM + m] * beta[(long long)m * B.Ncplx + k];
        gamma[i] = g;
    }
}

__device__ __forceinline__ double alpha_at(const double* __restrict__ alpha, int nmax, int lam, int iz, int iy, int ix) {
    const double* a = alpha + (long long)lam * 3 * nmax;
    return a[iz] * a[nmax + iy] * a[2 * nmax + ix];
}

// Small-P path (P <= 64).  Per-CTA partial sums of the upper triangle of [A y]^T [A y] (pairs
// (i, k), i <= k <= P), the columns formed 32 rows at a time in shared memory.  QPASS (pass 2 of
// CholeskyQR2): the staged A part of each row is first multiplied by R1^{-1} = L1^{-T} in place
// (eight threads per row, forward substitution), so the sums are those of [Q1 y].
template <bool QPASS>
__global__ void __launch_bounds__(256) k_fit_gram(const double* __restrict__ w, const float* __restrict__ y,
                                                  const double* __restrict__ alpha, int nmax, int p, BasisDev B,
                                                  const double* __restrict__ L1, double* __restrict__ partial) {
    const int P = B.P, PC = P + 1;
    const int npairs = PC * (PC + 1) / 2;
    __shared__ double cols[kGramRows][kMaxSmall + 1];
    __shared__ double wv[kGramRows][kMaxMult];
    __shared__ double av[kGramRows][kMaxSpatial];
    __shared__ unsigned short pi_[(kMaxSmall + 1) * (kMaxSmall + 2) / 2], pk_[(kMaxSmall + 1) * (kMaxSmall + 2) / 2];
    for (int t = threadIdx.x; t < npairs; t += blockDim.x) {
        int i = 0, rem = t;
        while (rem >= PC - i) {
            rem -= PC - i;
            ++i;
        }
        pi_[t] = (unsigned short)i;
        pk_[t] = (unsigned short)(i + rem);
    }
    constexpr int kMaxPairsPerThread = ((kMaxSmall + 1) * (kMaxSmall + 2) / 2 + 255) / 256;
    double acc[kMaxPairsPerThread];
#pragma unroll
    for (int s = 0; s < kMaxPairsPerThread; ++s) acc[s] = 0.0;
    const long long rows = (long long)p * B.npts;
    const long long wstride = (long long)p * B.Nreal;  // between multipliers
    const int tr = threadIdx.x >> 3, l8 = threadIdx.x & 7;  // pass 2: row and lane of the row solve
    __syncthreads();
    for (long long r0 = (long long)blockIdx.x * kGramRows; r0 < rows; r0 += (long long)gridDim.x * kGramRows) {
        // stage multiplier fields, spatial modes and y for kGramRows rows
        for (int t = threadIdx.x; t < kGramRows * (B.NM + B.nspatial + 1); t += blockDim.x) {
            const int r = t % kGramRows, c = t / kGramRows;
            const long long row = r0 + r;
            double v = 0.0;
            if (row < rows) {
                const int j = (int)(row / B.npts);
                const long long pt = row - (long long)j * B.npts;
                int iz, iy, ix;
                unravel(pt, B, iz, iy, ix);
                if (c < B.NM)
                    v = w[(long long)c * wstride + (long long)j * B.Nreal + fft_index(B, iz, iy, ix)];
                else if (c < B.NM + B.nspatial)
                    v = alpha_at(alpha, nmax, c - B.NM, iz, iy, ix);
                else
                    v = (double)y[row];
            }
            if (c < B.NM)
                wv[r][c] = v;
            else if (c < B.NM + B.nspatial)
                av[r][c - B.NM] = v;
            else
                cols[r][P] = v;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < kGramRows * P; t += blockDim.x) {
            const int r = t % kGramRows, i = t / kGramRows;
            const int lam = i / B.NM, m = i % B.NM;
            cols[r][i] = av[r][lam] * wv[r][m];
        }
        __syncthreads();
        if (QPASS) {  // q_j = (a_j - sum_{i<j} q_i L1_ji) / L1_jj for row tr, lanes l8 split the sum
            for (int jj = 0; jj < P; ++jj) {
                const double* Lj = L1 + (long long)jj * P;
                double sum = 0.0;
                for (int i = l8; i < jj; i += 8) sum = fma(cols[tr][i], Lj[i], sum);
                sum += __shfl_xor_sync(0xffffffffu, sum, 4);
                sum += __shfl_xor_sync(0xffffffffu, sum, 2);
                sum += __shfl_xor_sync(0xffffffffu, sum, 1);
                if (l8 == 0) cols[tr][jj] = (cols[tr][jj] - sum) / Lj[jj];
                __syncwarp();
            }
            __syncthreads();
        }
#pragma unroll
        for (int s = 0; s < kMaxPairsPerThread; ++s) {
            const int t = threadIdx.x + s * 256;
            if (t < npairs) {
                const int i = pi_[t], k = pk_[t];
                double a = acc[s];
#pragma unroll 8
                for (int r = 0; r < kGramRows; ++r) a = fma(cols[r][i], cols[r][k], a);
                acc[s] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < kMaxPairsPerThread; ++s) {
        const int t = threadIdx.x + s * 256;
        if (t < npairs) partial[(long long)blockIdx.x * npairs + t] = acc[s];
    }
}

// Small-P path: the per-CTA pair sums reduced in a fixed order into the dense lower triangle of
// C (n x n, n = P + 1, row-major): C[k][i] = sum (i <= k).
__global__ void k_fit_pairs_to_C(const double* __restrict__ partial, int nblocks, int n, double* __restrict__ C) {
    const int npairs = n * (n + 1) / 2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npairs; t += gridDim.x * blockDim.x) {
        int i = 0, rem = t;
        while (rem >= n - i) {
            rem -= n - i;
            ++i;
        }
        const int k = i + rem;
        double s = 0.0;
        for (int blk = 0; blk < nblocks; ++blk) s += partial[(long long)blk * npairs + t];
        C[(long long)k * n + i] = s;
    }
}

// [A | y] for stacked rows r0 .. r0 + rc - 1 (row = j * npts + pt) as a column-major FP64 block
// with leading dimension rc: column i < P is (B_i x_j)(pt) = alpha_lam(pt) w_m(j, pt) with
// i = lam * NM + m, column P is y_j(pt).  Rows past the end are zero (they add nothing).
__global__ void k_fit_cols(const double* __restrict__ w, const float* __restrict__ y,
                           const double* __restrict__ alpha, int nmax, int p, BasisDev B, long long r0, int rc,
                           double* __restrict__ A) {
    const long long rows = (long long)p * B.npts;
    const long long wstride = (long long)p * B.Nreal;
    const long long tot = (long long)rc * (B.P + 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(i / rc);
        const int r = (int)(i - (long long)col * rc);
        const long long row = r0 + r;
        double v = 0.0;
        if (row < rows) {
            const int j = (int)(row / B.npts);
            int iz, iy, ix;
            unravel(row - (long long)j * B.npts, B, iz, iy, ix);
            if (col < B.P) {
                const int lam = col / B.NM, m = col - lam * B.NM;
                v = alpha_at(alpha, nmax, lam, iz, iy, ix) *
                    w[(long long)m * wstride + (long long)j * B.Nreal + fft_index(B, iz, iy, ix)];
            } else {
                v = (double)y[row];
            }
        }
        A[i] = v;
    }
}

// Gram matrix of a column-major block A (rc rows, n columns, ld rc): tile (ti, tk), ti >= tk, of
// 64 x 64 entries over the rows of slice blockIdx.y; part[slice][i * n + k] for every (i, k) of
// the tile (the diagonal tiles hold both triangles).  256 threads, 4 x 4 entries each.
constexpr int kSyT = 64, kSyR = 32;
__global__ void __launch_bounds__(256) k_fit_syrk(const double* __restrict__ A, int rc, int n, int rows_per_slice,
                                                  double* __restrict__ part) {
    __shared__ double As[kSyR][kSyT + 1], Bs[kSyR][kSyT + 1];
    int t = blockIdx.x, ti = 0;
    while (t > ti) {  // lower tiles in row order: (0,0), (1,0), (1,1), (2,0), ...
        t -= ti + 1;
        ++ti;
    }
    const int tk = t;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r_beg = blockIdx.y * rows_per_slice, r_end = min(rc, r_beg + rows_per_slice);
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int r0 = r_beg; r0 < r_end; r0 += kSyR) {
        for (int q = threadIdx.x; q < kSyR * kSyT; q += 256) {
            const int r = q & (kSyR - 1), c = q / kSyR;
            const int row = r0 + r;
            const int ci = ti * kSyT + c, ck = tk * kSyT + c;
            As[r][c] = (row < r_end && ci < n) ? A[(long long)ci * rc + row] : 0.0;
            Bs[r][c] = (row < r_end && ck < n) ? A[(long long)ck * rc + row] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < kSyR; ++r) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[r][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[r][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
    double* out = part + (long long)blockIdx.y * n * n;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = ti * kSyT + ty * 4 + a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = tk * kSyT + tx * 4 + b;
            if (i < n && k < n) out[(long long)i * n + k] = acc[a][b];
        }
    }
}

// C[e] (+)= sum over slices of part[s][e] for the lower triangle, in slice order.
__global__ void k_fit_reduce(const double* __restrict__ part, int nslices, int n, int accumulate,
                             double* __restrict__ C) {
    const long long tot = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), k = (int)(e - (long long)i * n);
        if (k > i) continue;
        double s = accumulate ? C[e] : 0.0;
        for (int q = 0; q < nslices; ++q) s += part[(long long)q * tot + e];
        C[e] = s;
    }
}

// Largest diagonal entry of the leading P x P block of S (ld = ld) -> *dmax.
__global__ void k_fit_dmax(const double* __restrict__ S, int ld, int P, double* dmax) {
    double m = 0.0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) m = fmax(m, S[(long long)i * ld + i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        *dmax = m;
    }
}

// Step k of the right-looking Cholesky factorisation S = L L^T of the leading P x P block of S
// (lower triangle, ld = ld): CTA 0 writes column k of L (ld P); every CTA applies the rank-one
// update S_ij -= l_ik l_jk to its share of k < j <= i < P.  Column k of S is only read.  A pivot
// below 1e-13 of the largest diagonal entry marks S as not numerically positive definite.
__global__ void k_fit_chol_step(double* __restrict__ S, int ld, int P, int k, const double* __restrict__ dmax,
                                double* __restrict__ L, int* status) {
    const double d = S[(long long)k * ld + k];
    const bool bad = !(d > 1e-13 * (*dmax));
    const double lkk = bad ? 1.0 : sqrt(d);
    const double inv = 1.0 / lkk;
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            L[(long long)k * P + k] = lkk;
            if (bad) *status = 1;
        }
        for (int i = k + 1 + threadIdx.x; i < P; i += blockDim.x) L[(long long)i * P + k] = S[(long long)i * ld + k] * inv;
    }
    const int m = P - k - 1;
    const long long tot = (long long)m * m;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = k + 1 + (int)(t / m), j = k + 1 + (int)(t % m);
        if (j > i) continue;
        S[(long long)i * ld + j] -= (S[(long long)i * ld + k] * inv) * (S[(long long)j * ld + k] * inv);
    }
}

// Rows of a column-major block A (rc rows, first P columns) times R^{-1} = L^{-T}, in place:
// q_j = (a_j - sum_{i<j} q_i L_ji) / L_jj, one thread per row.
__global__ void k_fit_trsm_rows(double* __restrict__ A, int rc, int P, const double* __restrict__ L) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rc) return;
    for (int j = 0; j < P; ++j) {
        const double* Lj = L + (long long)j * P;
        double s = A[(long long)j * rc + r];
        for (int i = 0; i < j; ++i) s = fma(-A[(long long)i * rc + r], Lj[i], s);
        A[(long long)j * rc + r] = s / Lj[j];
    }
}

// One CTA: x = L^{-1} b (trans = 0) or x = L^{-T} b (trans = 1), L lower with ld P; x may alias b.
__global__ void __launch_bounds__(256) k_fit_trsv(const double* __restrict__ L, int P, int trans,
                                                  const double* b, double* x) {
    __shared__ double xs[kMaxTerms];
    __shared__ double red[8];
    for (int i = threadIdx.x; i < P; i += blockDim.x) xs[i] = b[i];
    __syncthreads();
    for (int s = 0; s < P; ++s) {
        const int i = trans ? P - 1 - s : s;
        double part = 0.0;
        if (!trans) {
            for (int j = threadIdx.x; j < i; j += blockDim.x) part = fma(L[(long long)i * P + j], xs[j], part);
        } else {
            for (int j = i + 1 + threadIdx.x; j < P; j += blockDim.x) part = fma(L[(long long)j * P + i], xs[j], part);
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            xs[i] = (xs[i] - t) / L[(long long)i * P + i];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) x[i] = xs[i];
}

// Per-CTA sums of (y - sum_i c_i col_i)^2 and y^2.
__global__ void __launch_bounds__(256) k_fit_resid(const double* __restrict__ w, const float* __restrict__ y,
                                                   const double* __restrict__ alpha, int nmax, int p, BasisDev B,
                                                   const double* __restrict__ coef, double* __restrict__ partial) {
    const long long rows = (long long)p * B.npts;
    const long long wstride = (long long)p * B.Nreal;
    double rr = 0.0, yy = 0.0;
    for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < rows;
         row += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(row / B.npts);
        int iz, iy, ix;
        unravel(row - (long long)j * B.npts, B, iz, iy, ix);
        const long long q = (long long)j * B.Nreal + fft_index(B, iz, iy, ix);
        double s = 0.0;
        for (int lam = 0; lam < B.nspatial; ++lam) {
            double t = 0.0;
            for (int m = 0; m < B.NM; ++m) t += coef[lam * B.NM + m] * w[(long long)m * wstride + q];
            s += alpha_at(alpha, nmax, lam, iz, iy, ix) * t;
        }
        const double yv = (double)y[row];
        rr += (yv - s) * (yv - s);
        yy += yv * yv;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        yy += __shfl_xor_sync(0xffffffffu, yy, o);
    }
    __shared__ double red[2][8];
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = rr;
        red[1][threadIdx.x >> 5] = yy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += red[0][i];
            c += red[1][i];
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = c;
    }
}

__global__ void k_fit_resid_final(const double* __restrict__ partial, int nblocks, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int i = 0; i < nblocks; ++i) {
            a += partial[2 * i];
            c += partial[2 * i + 1];
        }
        out[0] = c > 0.0 ? sqrt(a / c) : 0.0;
    }
}

// out(x) = sum_lam alpha_lam(x) w_lam(x) on the interior (FP32 result)
__global__ void k_precond_combine(const double* __restrict__ w, const double* __restrict__ alpha, int nmax, BasisDev B,
                                  float* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < B.npts;
         i += (long long)gridDim.x * blockDim.x) {
        int iz, iy, ix;
        unravel(i, B, iz, iy, ix);
        const long long q = fft_index(B, iz, iy, ix);
        double s = 0.0;
        for (int lam = 0; lam < B.nspatial; ++lam)
            s += alpha_at(alpha, nmax, lam, iz, iy, ix) * w[(long long)lam * B.Nreal + q];
        out[i] = (float)s;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

int grid_of(long long n, int cap = 152 * 16) {
    long long b = (n + 255) / 256;
    return (int)std::max(1LL, std::min<long long>(b, cap));
}

probe_status make_basis(probe_t h, const probe_basis* bs, BasisDev& B) {
    if (!bs) return fail(h, PROBE_ERR_ARG, "basis is NULL");
    if (bs->ndim != h->ndim) return fail(h, PROBE_ERR_ARG, "basis ndim differs from the grid's");
    if (bs->nspatial < 1 || bs->nspatial > kMaxSpatial || !bs->spatial)
        return fail(h, PROBE_ERR_ARG, "nspatial must be in [1, 32] with a spatial table");
    if (bs->nangular < 1 || bs->nangular > kMaxAngular || !bs->angular)
        return fail(h, PROBE_ERR_ARG, "nangular must be in [1, 16] with an angular table");
    if (bs->nradial < 1 || bs->nradial > kMaxRadial) return fail(h, PROBE_ERR_ARG, "nradial must be in [1, 16]");
    if (!(bs->L > 0) || !std::isfinite(bs->L)) return fail(h, PROBE_ERR_ARG, "L must be > 0");
    if (!std::isfinite(bs->order)) return fail(h, PROBE_ERR_ARG, "order must be finite");
    if (bs->fft_pad < 0 || bs->fft_pad > 4096) return fail(h, PROBE_ERR_ARG, "fft_pad out of range");
    memset(&B, 0, sizeof(B));
    B.ndim = h->ndim;
    B.n[0] = h->nz;
    B.n[1] = h->ndim == 3 ? h->ny : 1;
    B.n[2] = h->nx;
    B.h[0] = h->hz;
    B.h[1] = h->ndim == 3 ? h->hy : 1.0;
    B.h[2] = h->hx;
    B.fp = bs->fft_pad;
    B.Nf[0] = B.n[0] + 2 * B.fp;
    B.Nf[1] = h->ndim == 3 ? B.n[1] + 2 * B.fp : 1;
    B.Nf[2] = B.n[2] + 2 * B.fp;
    B.nspatial = bs->nspatial;
    B.nangular = bs->nangular;
    B.nradial = bs->nradial;
    B.NM = bs->nangular * bs->nradial;
    B.P = B.nspatial * B.NM;
    if (B.NM > kMaxMult) return fail(h, PROBE_ERR_ARG, "nangular * nradial must be <= 32");
    if (B.P > kMaxTerms) return fail(h, PROBE_ERR_ARG, "the number of terms P must be <= 1024");
    for (int l = 0; l < B.nspatial; ++l)
        for (int a = 0; a < bs->ndim; ++a) B.spatial[l][a] = bs->spatial[l * bs->ndim + a];
    for (int a = 0; a < B.nangular; ++a) {
        B.angular[a] = bs->angular[a];
        if (B.ndim == 3 && (B.angular[a] < 0 || B.angular[a] > 5))
            return fail(h, PROBE_ERR_ARG, "3D angular indices must be in [0, 5]");
    }
    B.L = bs->L;
    B.order = bs->order;
    B.Nreal = (long long)B.Nf[0] * B.Nf[1] * B.Nf[2];
    B.Ncplx = (long long)B.Nf[0] * B.Nf[1] * (B.Nf[2] / 2 + 1);
    B.npts = (long long)B.n[0] * B.n[1] * B.n[2];
    return PROBE_OK;
}

probe_status get_plan(probe_t h, const BasisDev& B, cufftType type, int batch, cudaStream_t st, cufftHandle* out) {
    if (!h->fit) h->fit = new FitCache();
    auto key = std::make_tuple(B.ndim, B.Nf[0], B.Nf[1], B.Nf[2], (type == CUFFT_D2Z ? 1 : 2) * 100000 + batch);
    auto it = h->fit->plans.find(key);
    cufftHandle plan;
    if (it == h->fit->plans.end()) {
        int n2[2] = {B.Nf[0], B.Nf[2]};
        int n3[3] = {B.Nf[0], B.Nf[1], B.Nf[2]};
        const int idist = (int)(type == CUFFT_D2Z ? B.Nreal : B.Ncplx);
        const int odist = (int)(type == CUFFT_D2Z ? B.Ncplx : B.Nreal);
        cufftResult r = cufftPlanMany(&plan, B.ndim, B.ndim == 2 ? n2 : n3, nullptr, 1, idist, nullptr, 1, odist,
                                      type, batch);
        if (r != CUFFT_SUCCESS) return fail(h, PROBE_ERR_CUDA, "cufftPlanMany failed (" + std::to_string((int)r) + ")");
        h->fit->plans[key] = plan;
    } else {
        plan = it->second;
    }
    if (cufftSetStream(plan, st) != CUFFT_SUCCESS) return fail(h, PROBE_ERR_CUDA, "cufftSetStream failed");
    *out = plan;
    return PROBE_OK;
}

probe_status fft_check(probe_t h, cufftResult r, const char* what) {
    if (r != CUFFT_SUCCESS) return fail(h, PROBE_ERR_CUDA, std::string(what) + " failed (" + std::to_string((int)r) + ")");
    return PROBE_OK;
}

// Stage an FP32 array of n elements on the device; returns the device pointer.
probe_status stage_f32(probe_t h, const float* p, size_t n, DevBuf& buf, const float** out, cudaStream_t st) {
    if (is_device_ptr(p)) {
        *out = p;
        return PROBE_OK;
    }
    PROBE_TRY(ensure_buf(h, buf, n * 4));
    PROBE_CK(h, cudaMemcpyAsync(buf.p, p, n * 4, cudaMemcpyHostToDevice, st));
    *out = (const float*)buf.p;
    return PROBE_OK;
}

// beta and alpha tables of a basis into the cache; returns pointers and nmax.
probe_status tables(probe_t h, const BasisDev& B, cudaStream_t st, double** beta, double** alpha, int* nmax) {
    FitCache& c = *h->fit;
    *nmax = std::max(B.n[0], std::max(B.n[1], B.n[2]));
    PROBE_TRY(ensure_buf(h, c.beta, (size_t)B.NM * B.Ncplx * 8));
    PROBE_TRY(ensure_buf(h, c.alpha, (size_t)B.nspatial * 3 * (*nmax) * 8));
    k_fit_beta<<<grid_of((long long)B.NM * B.Ncplx), 256, 0, st>>>((double*)c.beta.p, B);
    k_fit_alpha<<<grid_of((long long)B.nspatial * 3 * (*nmax)), 256, 0, st>>>((double*)c.alpha.p, B, *nmax);
    PROBE_CK(h, cudaGetLastError());
    *beta = (double*)c.beta.p;
    *alpha = (double*)c.alpha.p;
    return PROBE_OK;
}

// Gram matrix [A | y]^T [A | y] (pass 1) or [Q1 | y]^T [Q1 | y] with Q1 = A R1^{-1} (pass 2, L1 =
// R1^T given) into the dense lower triangle of C (n x n, n = P + 1).
probe_status fit_gram(probe_t h, const BasisDev& B, const double* w, const float* yd, const double* alpha, int nmax,
                      int p, const double* L1, double* C, cudaStream_t st) {
    FitCache& c = *h->fit;
    const int P = B.P, n = P + 1;
    const long long rows = (long long)p * B.npts;
    if (P <= kMaxSmall) {
        const int npairs = n * (n + 1) / 2;
        PROBE_TRY(ensure_buf(h, c.part, (size_t)kGramBlocks * npairs * 8));
        if (L1)
            k_fit_gram<true><<<kGramBlocks, 256, 0, st>>>(w, yd, alpha, nmax, p, B, L1, (double*)c.part.p);
        else
            k_fit_gram<false><<<kGramBlocks, 256, 0, st>>>(w, yd, alpha, nmax, p, B, nullptr, (double*)c.part.p);
        k_fit_pairs_to_C<<<grid_of(npairs), 256, 0, st>>>((const double*)c.part.p, kGramBlocks, n, C);
        PROBE_CK(h, cudaGetLastError());
        return PROBE_OK;
    }
    long long rcl = std::max<long long>(1024, kChunkBytes / (8ll * n));
    rcl = std::min(rcl, (rows + 31) / 32 * 32);
    const int rc = (int)((rcl + 31) / 32 * 32);
    const int T = (n + kSyT - 1) / kSyT, tiles = T * (T + 1) / 2;
    const int nslices = std::max(1, std::min(kGramBlocks / tiles, (rc + 255) / 256));
    const int rps = ((rc + nslices - 1) / nslices + kSyR - 1) / kSyR * kSyR;
    PROBE_TRY(ensure_buf(h, c.chunk, (size_t)rc * n * 8));
    PROBE_TRY(ensure_buf(h, c.part, (size_t)nslices * n * n * 8));
    double* A = (double*)c.chunk.p;
    for (long long r0 = 0; r0 < rows; r0 += rc) {
        k_fit_cols<<<grid_of((long long)rc * n), 256, 0, st>>>(w, yd, alpha, nmax, p, B, r0, rc, A);
        if (L1) k_fit_trsm_rows<<<(rc + 127) / 128, 128, 0, st>>>(A, rc, P, L1);
        k_fit_syrk<<<dim3(tiles, nslices), 256, 0, st>>>(A, rc, n, rps, (double*)c.part.p);
        k_fit_reduce<<<grid_of((long long)n * n), 256, 0, st>>>((const double*)c.part.p, nslices, n, r0 > 0 ? 1 : 0,
                                                               C);
        PROBE_CK(h, cudaGetLastError());
    }
    return PROBE_OK;
}

// Cholesky factor L (P x P, lower, ld P) of the leading block of C (ld n), destroying that block.
probe_status fit_cholesky(probe_t h, double* C, int n, int P, double* L, double* dmax, int* status,
                          cudaStream_t st) {
    PROBE_CK(h, cudaMemsetAsync(L, 0, (size_t)P * P * 8, st));
    k_fit_dmax<<<1, 256, 0, st>>>(C, n, P, dmax);
    for (int k = 0; k < P; ++k) {
        const long long m = (long long)(P - k - 1) * (P - k - 1);
        k_fit_chol_step<<<(int)std::max<long long>(1, std::min<long long>((m + 255) / 256, 1024)), 256, 0, st>>>(
            C, n, P, k, dmax, L, status);
    }
    PROBE_CK(h, cudaGetLastError());
    return PROBE_OK;
}

// CholeskyQR2 least squares of the fit: coefficients into coef (device, P); status[0] = 1 when
// A^T A (or Q1^T Q1) is not numerically positive definite.
probe_status fit_solve_cqr2(probe_t h, const BasisDev& B, const double* w, const float* yd, const double* alpha,
                            int nmax, int p, double* coef, int* status, cudaStream_t st) {
    FitCache& c = *h->fit;
    const int P = B.P, n = P + 1;
    PROBE_TRY(ensure_buf(h, c.gram, (size_t)n * n * 8));
    PROBE_TRY(ensure_buf(h, c.L1, (size_t)P * P * 8));
    PROBE_TRY(ensure_buf(h, c.L2, (size_t)P * P * 8));
    double* C = (double*)c.gram.p;
    double* L1 = (double*)c.L1.p;
    double* L2 = (double*)c.L2.p;
    double* dmax = (double*)c.misc.p + 2;
    double* v = coef + P;  // scratch of P doubles after the coefficients
    PROBE_CK(h, cudaMemsetAsync(status, 0, sizeof(int), st));
    PROBE_TRY(fit_gram(h, B, w, yd, alpha, nmax, p, nullptr, C, st));   // [A y]^T [A y]
    PROBE_TRY(fit_cholesky(h, C, n, P, L1, dmax, status, st));         // R1 = L1^T
    PROBE_TRY(fit_gram(h, B, w, yd, alpha, nmax, p, L1, C, st));        // [Q1 y]^T [Q1 y]
    PROBE_TRY(fit_cholesky(h, C, n, P, L2, dmax, status, st));         // R2 = L2^T
    const double* z = C + (long long)P * n;                             // Q1^T y (row P of C)
    k_fit_trsv<<<1, 256, 0, st>>>(L2, P, 0, z, v);                      // R2^{-T} z
    k_fit_trsv<<<1, 256, 0, st>>>(L2, P, 1, v, v);                      // R2^{-1} R2^{-T} z
    k_fit_trsv<<<1, 256, 0, st>>>(L1, P, 1, v, coef);                   // c = R1^{-1} (...)
    PROBE_CK(h, cudaGetLastError());
    return PROBE_OK;
}

}  // namespace
}  // namespace probe

using namespace probe;

extern "C" probe_status probe_fit(probe_t h, const probe_basis* basis, const float* y, const float* Hy, int p,
                                  double* coeffs, double* resid_rel, probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (p < 1) return fail(h, PROBE_ERR_ARG, "need at least one trial function");
    if (!y || !Hy || !coeffs) return fail(h, PROBE_ERR_ARG, "NULL array");
    BasisDev B;
    PROBE_TRY(make_basis(h, basis, B));
    cudaStream_t st = (cudaStream_t)stream;
    if (!h->fit) h->fit = new FitCache();
    FitCache& c = *h->fit;
    DevBuf ystage, xstage;
    const float *yd = nullptr, *xd = nullptr;
    probe_status s = PROBE_OK;
    do {
        if ((s = stage_f32(h, y, (size_t)p * B.npts, ystage, &yd, st)) != PROBE_OK) break;
        if ((s = stage_f32(h, Hy, (size_t)p * B.npts, xstage, &xd, st)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.xr, (size_t)p * B.Nreal * 8)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.Xc, (size_t)p * B.Ncplx * 16)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.Wc, (size_t)p * B.Ncplx * 16)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.w, (size_t)B.NM * p * B.Nreal * 8)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.coef, (size_t)(2 * B.P + 8) * 8)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.misc, 64)) != PROBE_OK) break;
        double *beta, *alpha;
        int nmax;
        if ((s = tables(h, B, st, &beta, &alpha, &nmax)) != PROBE_OK) break;
        cufftHandle fwd, inv;
        if ((s = get_plan(h, B, CUFFT_D2Z, p, st, &fwd)) != PROBE_OK) break;
        if ((s = get_plan(h, B, CUFFT_Z2D, p, st, &inv)) != PROBE_OK) break;
        cudaError_t e = cudaMemsetAsync(c.xr.p, 0, (size_t)p * B.Nreal * 8, st);
        if (e != cudaSuccess) { s = cuda_fail(h, e, "memset"); break; }
        k_fit_pad<<<grid_of((long long)p * B.npts), 256, 0, st>>>(xd, (double*)c.xr.p, p, B);
        if ((s = fft_check(h, cufftExecD2Z(fwd, (double*)c.xr.p, (cufftDoubleComplex*)c.Xc.p), "D2Z")) != PROBE_OK) break;
        const double invN = 1.0 / (double)B.Nreal;
        for (int m = 0; m < B.NM && s == PROBE_OK; ++m) {
            k_fit_mult<<<grid_of((long long)p * B.Ncplx), 256, 0, st>>>(
                (const double2*)c.Xc.p, beta + (long long)m * B.Ncplx, (double2*)c.Wc.p, 1, p, B.Ncplx, invN);
            s = fft_check(h, cufftExecZ2D(inv, (cufftDoubleComplex*)c.Wc.p, (double*)c.w.p + (long long)m * p * B.Nreal),
                          "Z2D");
        }
        if (s != PROBE_OK) break;
        int* status = (int*)c.misc.p;
        double* coef = (double*)c.coef.p;
        if ((s = fit_solve_cqr2(h, B, (const double*)c.w.p, yd, alpha, nmax, p, coef, status, st)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.part, (size_t)kGramBlocks * 2 * 8)) != PROBE_OK) break;
        k_fit_resid<<<kGramBlocks, 256, 0, st>>>((const double*)c.w.p, yd, alpha, nmax, p, B, coef, (double*)c.part.p);
        k_fit_resid_final<<<1, 32, 0, st>>>((const double*)c.part.p, kGramBlocks, (double*)c.misc.p + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) { s = cuda_fail(h, e, "fit kernels"); break; }
        int stat_h = 0;
        double res_h = 0.0;
        if ((e = cudaMemcpyAsync(&stat_h, status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&res_h, (double*)c.misc.p + 1, sizeof(double), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(coeffs, coef, (size_t)B.P * 8, cudaMemcpyDefault, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            s = cuda_fail(h, e, "fit result copy");
            break;
        }
        if (resid_rel) *resid_rel = res_h;
        if (stat_h) s = fail(h, PROBE_ERR_STATE, "the fit columns B_i x_j are numerically rank deficient");
    } while (0);
    cudaStreamSynchronize(st);
    if (ystage.p) cudaFree(ystage.p);
    if (xstage.p) cudaFree(xstage.p);
    return s;
}

extern "C" probe_status probe_apply_precond(probe_t h, const probe_basis* basis, const double* coeffs,
                                            const float* img, float* out, probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (!coeffs || !img || !out) return fail(h, PROBE_ERR_ARG, "NULL array");
    BasisDev B;
    PROBE_TRY(make_basis(h, basis, B));
    cudaStream_t st = (cudaStream_t)stream;
    if (!h->fit) h->fit = new FitCache();
    FitCache& c = *h->fit;
    DevBuf istage, ostage;
    const float* id = nullptr;
    probe_status s = PROBE_OK;
    const bool host_out = !is_device_ptr(out);
    do {
        if ((s = stage_f32(h, img, (size_t)B.npts, istage, &id, st)) != PROBE_OK) break;
        float* od = out;
        if (host_out) {
            if ((s = ensure_buf(h, ostage, (size_t)B.npts * 4)) != PROBE_OK) break;
            od = (float*)ostage.p;
        }
        if ((s = ensure_buf(h, c.xr, (size_t)B.Nreal * 8)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.Xc, (size_t)B.Ncplx * 16)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.Wc, (size_t)B.nspatial * B.Ncplx * 16)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.w, (size_t)B.nspatial * B.Nreal * 8)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.coef, (size_t)(2 * B.P + 8) * 8)) != PROBE_OK) break;
        if ((s = ensure_buf(h, c.part, (size_t)B.nspatial * B.Ncplx * 8)) != PROBE_OK) break;
        double *beta, *alpha;
        int nmax;
        if ((s = tables(h, B, st, &beta, &alpha, &nmax)) != PROBE_OK) break;
        cudaError_t e = cudaMemcpyAsync(c.coef.p, coeffs, (size_t)B.P * 8, cudaMemcpyDefault, st);
        if (e != cudaSuccess) { s = cuda_fail(h, e, "coefficient copy"); break; }
        cufftHandle fwd, inv;
        if ((s = get_plan(h, B, CUFFT_D2Z, 1, st, &fwd)) != PROBE_OK) break;
        if ((s = get_plan(h, B, CUFFT_Z2D, B.nspatial, st, &inv)) != PROBE_OK) break;
        if ((e = cudaMemsetAsync(c.xr.p, 0, (size_t)B.Nreal * 8, st)) != cudaSuccess) { s = cuda_fail(h, e, "memset"); break; }
        k_fit_pad<<<grid_of(B.npts), 256, 0, st>>>(id, (double*)c.xr.p, 1, B);
        if ((s = fft_check(h, cufftExecD2Z(fwd, (double*)c.xr.p, (cufftDoubleComplex*)c.Xc.p), "D2Z")) != PROBE_OK) break;
        double* gamma = (double*)c.part.p;
        k_precond_gamma<<<grid_of((long long)B.nspatial * B.Ncplx), 256, 0, st>>>(beta, (const double*)c.coef.p, gamma, B);
        k_fit_mult<<<grid_of((long long)B.nspatial * B.Ncplx), 256, 0, st>>>(
            (const double2*)c.Xc.p, gamma, (double2*)c.Wc.p, B.nspatial, 1, B.Ncplx, 1.0 / (double)B.Nreal);
        if ((s = fft_check(h, cufftExecZ2D(inv, (cufftDoubleComplex*)c.Wc.p, (double*)c.w.p), "Z2D")) != PROBE_OK) break;
        k_precond_combine<<<grid_of(B.npts), 256, 0, st>>>((const double*)c.w.p, alpha, nmax, B, od);
        if ((e = cudaGetLastError()) != cudaSuccess) { s = cuda_fail(h, e, "precond kernels"); break; }
        if (host_out) {
            if ((e = cudaMemcpyAsync(out, od, (size_t)B.npts * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess) {
                s = cuda_fail(h, e, "precond output copy");
                break;
            }
        }
    } while (0);
    if (istage.p || ostage.p) {
        cudaStreamSynchronize(st);
        if (istage.p) cudaFree(istage.p);
        if (ostage.p) cudaFree(ostage.p);
    }
    return s;
}
