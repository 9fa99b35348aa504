// Auxiliary device kernels: interior <-> padded layouts, the slowness grid
// s = dt^2/m, receiver sampling of the last time level, finiteness checks, the
// 16-bit checkpoint codec (per-plane absmax scale, round-to-nearest cast) and
// the reduction of shot-group images into the caller's model-space output.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace probe {

static inline int grid_for(long long n, int threads = 256, int cap = 152 * 32) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// padded linear index of interior cell (iz, iy, ix); 2D uses Ny = 1, ny = 1.
__device__ __forceinline__ long long pidx(int iz, int iy, int ix, int pad, int pady, int Ny, int P) {
    return ((long long)(iz + pad) * Ny + (iy + pady)) * P + (ix + pad);
}

__global__ void k_embed(const float* __restrict__ src, float* __restrict__ dst, int nb, int nz,
                        int ny, int nx, int pad, int pady, int Ny, int P, long long F, float scale) {
    const long long nint = (long long)nz * ny * nx;
    const long long total = nint * nb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / nint);
        long long r = i - (long long)b * nint;
        const int ix = (int)(r % nx);
        r /= nx;
        const int iy = (int)(r % ny);
        const int iz = (int)(r / ny);
        dst[(long long)b * F + pidx(iz, iy, ix, pad, pady, Ny, P)] = scale * src[i];
    }
}

cudaError_t launch_embed(const float* src_int, float* dst_pad, int nb, int nz, int nx, int ny,
                         int pad, int Nz, int Nx, int Ny, int P, long long F, float scale,
                         cudaStream_t st) {
    (void)Nz;
    (void)Nx;
    const int pady = (Ny > 1) ? pad : 0;
    const long long total = (long long)nb * nz * ny * nx;
    k_embed<<<grid_for(total), 256, 0, st>>>(src_int, dst_pad, nb, nz, ny, nx, pad, pady, Ny, P, F,
                                             scale);
    return cudaGetLastError();
}

// s = dt^2 / m on every padded cell: m inside the interior, edge-extended m0 in
// the sponge, zero on the row-pitch padding.
__global__ void k_make_s(const float* __restrict__ m_int, const float* __restrict__ m0_int,
                         float* __restrict__ s, int nz, int ny, int nx, int pad, int pady, int Nz,
                         int Ny, int Nx, int P, long long F, float dt2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < F;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % P);
        const long long zy = i / P;
        const int y = (int)(zy % Ny);
        const int z = (int)(zy / Ny);
        if (x >= Nx) {
            s[i] = 0.f;
            continue;
        }
        const int iz = z - pad, iy = y - pady, ix = x - pad;
        const bool inside = iz >= 0 && iz < nz && iy >= 0 && iy < ny && ix >= 0 && ix < nx;
        const int cz = min(max(iz, 0), nz - 1), cy = min(max(iy, 0), ny - 1),
                  cx = min(max(ix, 0), nx - 1);
        const long long j = ((long long)cz * ny + cy) * nx + cx;
        const float m = (inside && m_int) ? m_int[j] : m0_int[j];
        s[i] = dt2 / m;
    }
}

cudaError_t launch_make_s(const float* m_int, const float* m0_int, float* s_pad, int nz, int ny,
                          int nx, int pad, int P, long long F, int Nz, int Ny, int Nx, float dt2,
                          cudaStream_t st) {
    const int pady = (Ny > 1) ? pad : 0;
    k_make_s<<<grid_for(F), 256, 0, st>>>(m_int, m0_int, s_pad, nz, ny, nx, pad, pady, Nz, Ny, Nx,
                                          P, F, dt2);
    return cudaGetLastError();
}

// out[b][interior] (+)= sum_g (img[g][b] - comp[g][b]), summed in FP64.
__global__ void k_extract(const float* __restrict__ img, const float* __restrict__ comp, int ngroups,
                          long long gstride, int nb, long long F, float* __restrict__ out, int nz,
                          int ny, int nx, int pad, int pady, int Ny, int P, int kahan, int accumulate) {
    const long long nint = (long long)nz * ny * nx;
    const long long total = nint * nb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / nint);
        long long r = i - (long long)b * nint;
        const int ix = (int)(r % nx);
        r /= nx;
        const int iy = (int)(r % ny);
        const int iz = (int)(r / ny);
        const long long q = (long long)b * F + pidx(iz, iy, ix, pad, pady, Ny, P);
        double acc = 0.0;
        for (int g = 0; g < ngroups; ++g) {
            acc += (double)img[g * gstride + q];
            if (kahan) acc -= (double)comp[g * gstride + q];
        }
        if (accumulate) acc += (double)out[i];
        out[i] = (float)acc;
    }
}

cudaError_t launch_extract_images(const float* img, const float* comp, int ngroups,
                                  long long group_stride, int nb, long long F, float* out, int nz,
                                  int ny, int nx, int pad, int Ny, int P, bool kahan,
                                  bool accumulate, cudaStream_t st) {
    const int pady = (Ny > 1) ? pad : 0;
    const long long total = (long long)nb * nz * ny * nx;
    k_extract<<<grid_for(total), 256, 0, st>>>(img, comp, ngroups, group_stride, nb, F, out, nz, ny,
                                               nx, pad, pady, Ny, P, kahan ? 1 : 0,
                                               accumulate ? 1 : 0);
    return cudaGetLastError();
}

// data[shot][trial][n][r] = field plane at receiver r.
__global__ void k_sample(const float* __restrict__ field, long long pss, long long pst, int plane,
                         long long F, int nshots, int nb, const int* __restrict__ rec, int nr, int P,
                         int ndim, int Ny, float* __restrict__ data, long long dss, long long dst_,
                         int n) {
    const long long total = (long long)nshots * nb * nr;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i % nr);
        const long long sb = i / nr;
        const int b = (int)(sb % nb);
        const int s = (int)(sb / nb);
        long long cell;
        if (ndim == 2)
            cell = (long long)rec[2 * r] * P + rec[2 * r + 1];
        else
            cell = ((long long)rec[3 * r] * Ny + rec[3 * r + 1]) * P + rec[3 * r + 2];
        const float v = field[s * pss + b * pst + (long long)plane * F + cell];
        data[s * dss + b * dst_ + (long long)n * nr + r] = v;
    }
}

// Adjoint receiver injection R^T r^n for `nsteps` time levels, scattered into the compact
// band buffer (the grid rows that hold receivers): one thread per (receiver cell, step, shot,
// trial) sums that cell's receivers in their list order (no atomics, so the result is the
// same on every run) and stores it at band * P + x of its (slot, shot, trial) block.  Slot
// k holds time level n_hi - k.  Cells without receivers stay as the caller zeroed them.
__global__ void k_build_injection(const float* __restrict__ rdata, long long dss, long long dts, int nr,
                                  int n_hi, int nsteps, int nshots, int nb, int nuc,
                                  const int* __restrict__ uc_ptr, const int* __restrict__ uc_rec,
                                  const int* __restrict__ uc_pos, float* __restrict__ inj, long long block) {
    const long long total = (long long)nuc * nsteps * nshots * nb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % nuc);
        long long r = i / nuc;
        const int b = (int)(r % nb);
        r /= nb;
        const int s = (int)(r % nshots);
        const int k = (int)(r / nshots);
        const int n = n_hi - k;
        const float* row = rdata + s * dss + b * dts + (long long)n * nr;
        float v = 0.f;
        for (int q = uc_ptr[c]; q < uc_ptr[c + 1]; ++q) v += row[uc_rec[q]];
        inj[(((long long)k * nshots + s) * nb + b) * block + uc_pos[c]] = v;
    }
}

cudaError_t launch_build_injection(const float* rdata, long long dss, long long dts, int nr, int n_hi, int nsteps,
                                   int nshots, int nb, int nuc, const int* uc_ptr, const int* uc_rec,
                                   const int* uc_pos, float* inj, long long block, cudaStream_t st) {
    const long long total = (long long)nuc * nsteps * nshots * nb;
    if (total <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)std::min<long long>((total + threads - 1) / threads, 65535);
    k_build_injection<<<blocks, threads, 0, st>>>(rdata, dss, dts, nr, n_hi, nsteps, nshots, nb, nuc, uc_ptr, uc_rec,
                                                   uc_pos, inj, block);
    return cudaGetLastError();
}

cudaError_t launch_sample(const float* field, long long plane_stride_shot,
                          long long plane_stride_trial, int plane, long long F, int nshots, int nb,
                          const int* rec_zx, int nr, int P, int ndim, int Ny, float* data,
                          long long data_shot_stride, long long data_trial_stride, int n,
                          cudaStream_t st) {
    const long long total = (long long)nshots * nb * nr;
    k_sample<<<grid_for(total), 256, 0, st>>>(field, plane_stride_shot, plane_stride_trial, plane, F,
                                              nshots, nb, rec_zx, nr, P, ndim, Ny, data,
                                              data_shot_stride, data_trial_stride, n);
    return cudaGetLastError();
}

__global__ void k_check_finite(const float* __restrict__ a, long long n, int* err) {
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(a[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_dev_error(err, DEVERR_NONFINITE);
}

cudaError_t launch_check_finite(const float* a, long long n, int* err, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_check_finite<<<grid_for(n), 256, 0, st>>>(a, n, err);
    return cudaGetLastError();
}

// ---- checkpoint codec ------------------------------------------------------
// A checkpoint holds, per shot, the leapfrog state (u^n, u^{n-1}).  In 16-bit
// storage it is kept as q0 = u^n and q1 = u^n - u^{n-1}, each with its own
// absmax scale: the time difference is much smaller than u itself, so
// quantising it separately keeps the restored state's time derivative accurate
// (independent rounding of u^n and u^{n-1} would leave an error of the size of
// u's rounding in their difference).  State plane 2j + pc holds u^n of shot j,
// plane 2j + (1 - pc) holds u^{n-1}.
//
// Storage planes per shot: FP16 keeps q0 and q1 (2 planes).  BF16 keeps q0 as
// the unevaluated sum of two BF16 numbers hi + lo (lo = the BF16 rounding of
// q0 - hi) and q1 as one (3 planes).  The reason: one BF16 number carries 8
// significant bits, and the rounding error of the restored position plane is
// white at the grid scale, where the 8th-order Laplacian multiplies it by up to
// sum|w_k| / h^2 per axis -- about 15 times the Dtt u of a field sampled at ten
// points per wavelength -- in every recomputed step of the segment.  With a
// single BF16 position plane the imaging result is off by about 1e-2; the
// two-term position plane (16 significant bits) leaves the rounding of q1,
// which is 10-20 times smaller in absolute size, as the dominant term.
struct CkptPlanes {
    int pps, p_un, p_prev;  // planes per shot; planes of u^n and u^{n-1} within a shot's block
};

__device__ __forceinline__ float ckpt_value(const float* __restrict__ state, long long F, int plane,
                                            CkptPlanes q, long long i) {
    const int shot = plane >> 1;
    const float un = state[(long long)(q.pps * shot + q.p_un) * F + i];
    if ((plane & 1) == 0) return un;
    return un - state[(long long)(q.pps * shot + q.p_prev) * F + i];
}

__global__ void k_absmax(const float* __restrict__ state, long long F, CkptPlanes pc, float* absmax) {
    const int plane = blockIdx.y;
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < F;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(ckpt_value(state, F, plane, pc, i)));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        atomicMax(reinterpret_cast<int*>(absmax + plane), __float_as_int(m));  // m >= 0
    }
}

// Scale so that |v| / scale <= 2^14 for FP16 (headroom below 65504) and <= 1 for BF16.
__device__ __forceinline__ float ckpt_scale(float amax, int dtype) {
    if (!(amax > 0.f)) return 1.f;
    return dtype == PROBE_SNAP_FP16 ? amax * (1.0f / 16384.0f) : amax;
}

__host__ __device__ constexpr int ckpt_store_planes(int dtype) {
    return dtype == PROBE_SNAP_BF16 ? 3 : 2;
}

size_t ckpt_bytes_per_shot(int dtype, long long F) {
    return (size_t)ckpt_store_planes(dtype) * (size_t)F * (dtype == PROBE_SNAP_FP32 ? 4u : 2u);
}

// blockIdx.y = logical plane (2 j + 0: q0 of shot j, 2 j + 1: q1).
__global__ void k_encode(const float* __restrict__ state, long long F, CkptPlanes pc, void* dst,
                         const float* __restrict__ absmax, float* scales, int dtype) {
    const int plane = blockIdx.y;
    const int shot = plane >> 1, which = plane & 1;
    const float sc = ckpt_scale(absmax[plane], dtype);
    const float inv = 1.0f / sc;
    if (blockIdx.x == 0 && threadIdx.x == 0) scales[plane] = sc;
    const long long base = (long long)shot * ckpt_store_planes(dtype) * F;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < F;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = __fmul_rn(ckpt_value(state, F, plane, pc, i), inv);
        if (dtype == PROBE_SNAP_FP16) {
            reinterpret_cast<__half*>(dst)[base + which * F + i] = __float2half_rn(v);
        } else {
            __nv_bfloat16* q = reinterpret_cast<__nv_bfloat16*>(dst) + base;
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            if (which == 0) {
                q[i] = hi;  // v - hi is exact in FP32
                q[F + i] = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(hi)));
            } else {
                q[2 * F + i] = hi;
            }
        }
    }
}

// blockIdx.y = shot: restores u^n and u^{n-1} into the shot's planes p_un and p_prev.
__global__ void k_decode(const void* src, const float* __restrict__ scales, long long F, int dtype,
                         CkptPlanes pc, float* __restrict__ state) {
    const int shot = blockIdx.y;
    const float s0 = scales[2 * shot], s1 = scales[2 * shot + 1];
    const long long base = (long long)shot * ckpt_store_planes(dtype) * F;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < F;
         i += (long long)gridDim.x * blockDim.x) {
        float q0, q1;
        if (dtype == PROBE_SNAP_FP16) {
            const __half* q = reinterpret_cast<const __half*>(src) + base;
            q0 = __half2float(q[i]);
            q1 = __half2float(q[F + i]);
        } else {
            const __nv_bfloat16* q = reinterpret_cast<const __nv_bfloat16*>(src) + base;
            q0 = __fadd_rn(__bfloat162float(q[i]), __bfloat162float(q[F + i]));  // exact: 17 bits
            q1 = __bfloat162float(q[2 * F + i]);
        }
        const float un = __fmul_rn(q0, s0);
        const float du = __fmul_rn(q1, s1);
        state[(long long)(pc.pps * shot + pc.p_un) * F + i] = un;
        state[(long long)(pc.pps * shot + pc.p_prev) * F + i] = __fsub_rn(un, du);
    }
}

// FP32 checkpoints: (u^n, u^{n-1}) of each shot copied as they are, u^n first.
__global__ void k_copy_pair(const float* __restrict__ state, long long F, CkptPlanes q, float* __restrict__ dst,
                            int to_state) {
    const int plane = blockIdx.y;  // 2 shot + (0: u^n, 1: u^{n-1})
    const int shot = plane >> 1;
    const long long sp = (long long)(q.pps * shot + ((plane & 1) ? q.p_prev : q.p_un)) * F;
    const long long cp = (long long)plane * F;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < F;
         i += (long long)gridDim.x * blockDim.x) {
        if (to_state)
            const_cast<float*>(state)[sp + i] = dst[cp + i];
        else
            dst[cp + i] = state[sp + i];
    }
}

cudaError_t launch_encode_ckpt(const float* state, int nplanes, long long F, int pps, int p_un, int p_prev, void* dst,
                               float* scales, int dtype, float* absmax_scratch, cudaStream_t st) {
    const CkptPlanes pc{pps, p_un, p_prev};
    if (dtype == PROBE_SNAP_FP32) {
        if (pps == 2 && p_un == 0 && p_prev == 1)  // already in checkpoint order
            return cudaMemcpyAsync(dst, state, (size_t)nplanes * F * sizeof(float), cudaMemcpyDeviceToDevice, st);
        k_copy_pair<<<dim3(grid_for(F, 256, 64), nplanes), 256, 0, st>>>(state, F, pc, (float*)dst, 0);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(absmax_scratch, 0, nplanes * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const int bx = grid_for(F, 256, 64);
    k_absmax<<<dim3(bx, nplanes), 256, 0, st>>>(state, F, pc, absmax_scratch);
    k_encode<<<dim3(bx, nplanes), 256, 0, st>>>(state, F, pc, dst, absmax_scratch, scales, dtype);
    return cudaGetLastError();
}

cudaError_t launch_decode_ckpt(const void* src, const float* scales, int nplanes, long long F, int pps, int p_un,
                               int p_prev, int dtype, float* state, cudaStream_t st) {
    const CkptPlanes pc{pps, p_un, p_prev};
    if (dtype == PROBE_SNAP_FP32) {
        if (pps == 2 && p_un == 0 && p_prev == 1)
            return cudaMemcpyAsync(state, src, (size_t)nplanes * F * sizeof(float), cudaMemcpyDeviceToDevice, st);
        k_copy_pair<<<dim3(grid_for(F, 256, 64), nplanes), 256, 0, st>>>(state, F, pc, (float*)src, 1);
        return cudaGetLastError();
    }
    const int bx = grid_for(F, 256, 64);
    k_decode<<<dim3(bx, nplanes / 2), 256, 0, st>>>(src, scales, F, dtype, pc, state);
    return cudaGetLastError();
}

__global__ void k_scale_copy(const float* __restrict__ src, float* __restrict__ dst, long long n,
                             float a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = a * src[i];
}

cudaError_t launch_scale_copy(const float* src, float* dst, long long n, float a, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_scale_copy<<<grid_for(n), 256, 0, st>>>(src, dst, n, a);
    return cudaGetLastError();
}

__global__ void k_kahan_fold(float4* __restrict__ img, float4* __restrict__ comp, const float4* __restrict__ seg,
                             long long n4) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        float4 s = img[i], c = comp[i];
        const float4 v = seg[i];
        kahan4(s, c, v.x, v.y, v.z, v.w);
        img[i] = s;
        comp[i] = c;
    }
}

cudaError_t launch_kahan_fold(float* img, float* comp, const float* seg, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n % 4) return cudaErrorInvalidValue;  // whole planes of a padded grid (pitch a multiple of 32)
    k_kahan_fold<<<grid_for(n / 4), 256, 0, st>>>(reinterpret_cast<float4*>(img), reinterpret_cast<float4*>(comp),
                                                   reinterpret_cast<const float4*>(seg), n / 4);
    return cudaGetLastError();
}

// Diagnostic: one CTA waits on an mbarrier phase that nothing ever completes, so
// the bounded wait can only end by its time limit; the kernel then records the
// timeout in the device error word and returns (the context stays usable).
__global__ void k_diag_wait(int* err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (!ok && threadIdx.x == 0) set_dev_error(err, DEVERR_TIMEOUT);
}

cudaError_t launch_diag_wait(int* err, unsigned long long limit_ns, cudaStream_t st) {
    k_diag_wait<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

}  // namespace probe
