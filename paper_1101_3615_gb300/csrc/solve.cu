// Iterative solution of the linearised least-squares problem through its normal equations
// H dm = F*d (Sec. 2: the fitted preconditioners are compared with gradient-descent iterations
// on 1/2 ||F dm - d||^2; preconditioned iterations apply the approximate inverse to the
// migrated residual).  Steepest descent with exact line search (optionally along the
// preconditioned residual) and conjugate gradients.  Every H application is probe_apply_H on
// one trial, every preconditioner application probe_apply_precond; the vector updates and the
// FP64 inner products are the kernels of this file.
#include <cmath>
#include <string>

#include "common.cuh"
#include "handle.h"
#include "internal.h"

namespace probe {

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 304;  // two CTAs per SM; the partial sums are reduced by one CTA
constexpr int kMaxDots = 2;

// Block-level tree sum of one double per thread; the result is in sh[0].
__device__ __forceinline__ void block_sum(double* sh) {
    __syncthreads();
    for (int s = kDotThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
}

// partial[d * gridDim.x + block] = sum over the block's elements of a_d[i] b_d[i] (FP64), for
// the ndot pairs (a_d, b_d).  Fixed element-to-thread map and reduction order: deterministic.
struct DotArgs {
    const float* a[kMaxDots];
    const float* b[kMaxDots];
};
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(DotArgs args, int ndot, long long n, double* partial) {
    __shared__ double sh[kDotThreads];
    for (int d = 0; d < ndot; ++d) {
        const float* a = args.a[d];
        const float* b = args.b[d];
        double acc = 0.0;
        for (long long i = (long long)blockIdx.x * kDotThreads + threadIdx.x; i < n;
             i += (long long)gridDim.x * kDotThreads)
            acc = fma((double)a[i], (double)b[i], acc);
        sh[threadIdx.x] = acc;
        block_sum(sh);
        if (threadIdx.x == 0) partial[d * gridDim.x + blockIdx.x] = sh[0];
        __syncthreads();
    }
}

// out[d] = sum of the nblocks partial sums of dot d (one CTA, fixed order).
__global__ void __launch_bounds__(kDotThreads) k_dot_final(const double* partial, int ndot, int nblocks, double* out) {
    __shared__ double sh[kDotThreads];
    for (int d = 0; d < ndot; ++d) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < nblocks; i += kDotThreads) acc += partial[d * nblocks + i];
        sh[threadIdx.x] = acc;
        block_sum(sh);
        if (threadIdx.x == 0) out[d] = sh[0];
        __syncthreads();
    }
}

// x += alpha p and r -= alpha Hp (one pass over the four vectors).
__global__ void k_step_update(float* x, float* r, const float* p, const float* Hp, float alpha, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] = __fmaf_rn(alpha, p[i], x[i]);
        r[i] = __fmaf_rn(-alpha, Hp[i], r[i]);
    }
}

// p = z + beta p.
__global__ void k_direction(float* p, const float* z, float beta, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = __fmaf_rn(beta, p[i], z[i]);
}

// y = x / sqrt(*sumsq) (y = 0 when the norm is zero); the norm is read on the device.
__global__ void k_scale_by_norm(float* y, const float* x, const double* sumsq, long long n) {
    const double s = *sumsq;
    const float inv = (s > 0.0) ? (float)(1.0 / sqrt(s)) : 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __fmul_rn(x[i], inv);
}

// r = rhs - Hx.
__global__ void k_residual(float* r, const float* rhs, const float* Hx, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = __fsub_rn(rhs[i], Hx[i]);
}

namespace {

int vec_grid(long long n) { return (int)std::min<long long>((n + 255) / 256, 152 * 8); }

struct SolveBufs {
    float *x = nullptr, *r = nullptr, *p = nullptr, *Hp = nullptr, *z = nullptr, *rhs = nullptr;
    double *partial = nullptr, *dots = nullptr;
    void release() {
        for (float* q : {x, r, p, Hp, z, rhs})
            if (q) cudaFree(q);
        if (partial) cudaFree(partial);
        if (dots) cudaFree(dots);
    }
};

// FP64 inner products of ndot pairs, copied to host vals (synchronises st).
probe_status dots(probe_t h, const SolveBufs& b, int ndot, const float* const* a, const float* const* c, long long n,
                  cudaStream_t st, double* vals) {
    DotArgs args{};
    for (int d = 0; d < ndot; ++d) {
        args.a[d] = a[d];
        args.b[d] = c[d];
    }
    k_dot_partial<<<kDotBlocks, kDotThreads, 0, st>>>(args, ndot, n, b.partial);
    k_dot_final<<<1, kDotThreads, 0, st>>>(b.partial, ndot, kDotBlocks, b.dots);
    PROBE_CK(h, cudaGetLastError());
    PROBE_CK(h, cudaMemcpyAsync(vals, b.dots, (size_t)ndot * 8, cudaMemcpyDeviceToHost, st));
    PROBE_CK(h, cudaStreamSynchronize(st));
    return PROBE_OK;
}

probe_status run_solve(probe_t h, int method, int iters, const probe_basis* basis, const double* coeffs,
                       SolveBufs& b, long long n, double* resid, int* done, cudaStream_t st) {
    const int grid = vec_grid(n);
    double v[kMaxDots];
    // r_0 = rhs - H x_0
    PROBE_TRY(probe_apply_H(h, b.x, b.Hp, 1, st));
    k_residual<<<grid, 256, 0, st>>>(b.r, b.rhs, b.Hp, n);
    PROBE_CK(h, cudaGetLastError());
    {
        const float* a[1] = {b.r};
        PROBE_TRY(dots(h, b, 1, a, a, n, st, v));
    }
    double rr = v[0];
    if (resid) resid[0] = std::sqrt(rr);
    int k = 0;
    if (method == PROBE_SOLVE_CG)
        PROBE_CK(h, cudaMemcpyAsync(b.p, b.r, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    for (; k < iters; ++k) {
        if (rr == 0.0) break;
        double alpha;
        if (method == PROBE_SOLVE_GD) {
            // direction p = M r_k (or r_k); exact line search alpha = p.r / p.Hp
            const float* dir = b.r;
            if (basis) {
                PROBE_TRY(probe_apply_precond(h, basis, coeffs, b.r, b.z, st));
                dir = b.z;
            }
            PROBE_TRY(probe_apply_H(h, dir, b.Hp, 1, st));
            const float* a[2] = {dir, dir};
            const float* c[2] = {b.r, b.Hp};
            PROBE_TRY(dots(h, b, 2, a, c, n, st, v));
            if (!(v[1] > 0.0)) break;
            alpha = v[0] / v[1];
            k_step_update<<<grid, 256, 0, st>>>(b.x, b.r, dir, b.Hp, (float)alpha, n);
            PROBE_CK(h, cudaGetLastError());
            const float* a1[1] = {b.r};
            PROBE_TRY(dots(h, b, 1, a1, a1, n, st, v));
            rr = v[0];
        } else {
            PROBE_TRY(probe_apply_H(h, b.p, b.Hp, 1, st));
            const float* a[1] = {b.p};
            const float* c[1] = {b.Hp};
            PROBE_TRY(dots(h, b, 1, a, c, n, st, v));
            if (!(v[0] > 0.0)) break;
            alpha = rr / v[0];
            k_step_update<<<grid, 256, 0, st>>>(b.x, b.r, b.p, b.Hp, (float)alpha, n);
            PROBE_CK(h, cudaGetLastError());
            const float* a1[1] = {b.r};
            PROBE_TRY(dots(h, b, 1, a1, a1, n, st, v));
            const double rr_new = v[0];
            k_direction<<<grid, 256, 0, st>>>(b.p, b.r, (float)(rr_new / rr), n);
            PROBE_CK(h, cudaGetLastError());
            rr = rr_new;
        }
        if (resid) resid[k + 1] = std::sqrt(rr);
    }
    if (done) *done = k;
    return PROBE_OK;
}

}  // namespace
}  // namespace probe

using namespace probe;

extern "C" probe_status probe_solve(probe_t h, int method, int iters, const probe_basis* basis, const double* coeffs,
                                    const float* rhs, float* x, double* resid, int* done, probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (method != PROBE_SOLVE_GD && method != PROBE_SOLVE_CG)
        return fail(h, PROBE_ERR_ARG, "method must be PROBE_SOLVE_GD or PROBE_SOLVE_CG");
    if (iters < 0) return fail(h, PROBE_ERR_ARG, "iters must be >= 0");
    if (!rhs || !x) return fail(h, PROBE_ERR_ARG, "NULL array");
    if ((basis == nullptr) != (coeffs == nullptr)) return fail(h, PROBE_ERR_ARG, "basis and coeffs go together");
    if (basis && method != PROBE_SOLVE_GD) return fail(h, PROBE_ERR_ARG, "a preconditioner needs PROBE_SOLVE_GD");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = h->nmodel;
    SolveBufs b;
    auto alloc = [&](void** q, size_t bytes) { return cudaMalloc(q, bytes); };
    cudaError_t e = cudaSuccess;
    for (float** q : {&b.x, &b.r, &b.p, &b.Hp, &b.rhs})
        if (e == cudaSuccess) e = alloc((void**)q, (size_t)n * 4);
    if (e == cudaSuccess && basis) e = alloc((void**)&b.z, (size_t)n * 4);
    if (e == cudaSuccess) e = alloc((void**)&b.partial, (size_t)kMaxDots * kDotBlocks * 8);
    if (e == cudaSuccess) e = alloc((void**)&b.dots, (size_t)kMaxDots * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.rhs, rhs, (size_t)n * 4, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.x, x, (size_t)n * 4, cudaMemcpyDefault, st);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        b.release();
        return cuda_fail(h, e, "solver buffers");
    }
    probe_status s = run_solve(h, method, iters, basis, coeffs, b, n, resid, done, st);
    if (s == PROBE_OK) {
        e = cudaMemcpyAsync(x, b.x, (size_t)n * 4, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(h, e, "solver result copy");
    } else {
        cudaStreamSynchronize(st);
    }
    b.release();
    return s;
}

// Krylov trial functions of the Kn preconditioners (Sec. 2): y_1 = rhs / ||rhs||, x_j = H y_j,
// y_{j+1} = x_j / ||x_j||.  The norms are FP64 sums on the device; nothing is read back between
// the H applications.
extern "C" probe_status probe_krylov_trials(probe_t h, const float* rhs, int n, float* y, float* Hy,
                                            probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (n < 1) return fail(h, PROBE_ERR_ARG, "n must be >= 1");
    if (!rhs || !y || !Hy) return fail(h, PROBE_ERR_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    const long long m = h->nmodel;
    const bool dev_y = is_device_ptr(y), dev_x = is_device_ptr(Hy);
    float *yd = dev_y ? y : nullptr, *xd = dev_x ? Hy : nullptr, *rd = nullptr;
    double *partial = nullptr, *sums = nullptr;
    cudaError_t e = cudaSuccess;
    if (!dev_y) e = cudaMalloc((void**)&yd, (size_t)n * m * 4);
    if (e == cudaSuccess && !dev_x) e = cudaMalloc((void**)&xd, (size_t)n * m * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&rd, (size_t)m * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&partial, (size_t)kDotBlocks * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sums, 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rd, rhs, (size_t)m * 4, cudaMemcpyDefault, st);
    probe_status s = (e == cudaSuccess) ? PROBE_OK : cuda_fail(h, e, "Krylov trial buffers");
    const int grid = vec_grid(m);
    for (int j = 0; j < n && s == PROBE_OK; ++j) {
        const float* src = (j == 0) ? rd : xd + (long long)(j - 1) * m;
        DotArgs args{};
        args.a[0] = src;
        args.b[0] = src;
        k_dot_partial<<<kDotBlocks, kDotThreads, 0, st>>>(args, 1, m, partial);
        k_dot_final<<<1, kDotThreads, 0, st>>>(partial, 1, kDotBlocks, sums);
        k_scale_by_norm<<<grid, 256, 0, st>>>(yd + (long long)j * m, src, sums, m);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            s = cuda_fail(h, e, "Krylov normalisation");
            break;
        }
        s = probe_apply_H(h, yd + (long long)j * m, xd + (long long)j * m, 1, stream);
    }
    if (s == PROBE_OK && !dev_y) e = cudaMemcpyAsync(y, yd, (size_t)n * m * 4, cudaMemcpyDeviceToHost, st);
    if (s == PROBE_OK && e == cudaSuccess && !dev_x)
        e = cudaMemcpyAsync(Hy, xd, (size_t)n * m * 4, cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (s == PROBE_OK && (e != cudaSuccess || e2 != cudaSuccess))
        s = cuda_fail(h, e != cudaSuccess ? e : e2, "Krylov trial copy");
    if (!dev_y && yd) cudaFree(yd);
    if (!dev_x && xd) cudaFree(xd);
    if (rd) cudaFree(rd);
    if (partial) cudaFree(partial);
    if (sums) cudaFree(sums);
    return s;
}
