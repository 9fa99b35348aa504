// 3D time-stepping kernels (sm_103a): incident step, Born step, adjoint step
// with imaging, one field per CTA.
//
// A CTA of 256 threads owns a 64 (x) x 16 (y) column tile and marches through
// ZC consecutive z planes.  The halo'd plane tiles (72 x 24 floats) of the
// field being differentiated stream through a ring of kRing shared-memory
// slots, each filled by one 4D TMA tiled load (x, y, z, volume) that completes
// on the slot's mbarrier; planes outside the grid read as zero (the zero
// extension of the Laplacian).  All 25 taps of the 8th-order Laplacian come
// from the ring: x and y taps from the current plane, z taps from the same
// column of the neighbouring planes.  Each thread updates 4 consecutive x
// cells (float4 I/O).  Scheme and adjoint form as in the 2D kernels:
//   incident  u^{n+1}  = G [2u^n  - a- u^{n-1}  + s (L u^n + f^n)], writes Dtt u^n
//   Born      du^{n+1} = G [2du^n - a- du^{n-1} + s (L du^n - dm Dtt u^n)]
//   adjoint   mu^n     = G [2mu^{n+1} - a- mu^{n+2} + s (L mu^{n+1} + R^T r^n)],
//             img -= Dtt u^{n-1} mu^n
#include "common.cuh"
#include "internal.h"

namespace probe {

constexpr int kTY3 = kTY3D;
constexpr int kRing = 10;
constexpr int kHX3 = kTX + 8;   // 72
constexpr int kHY3 = kTY3 + 8;  // 24
constexpr int kPlane3 = kHX3 * kHY3;
constexpr unsigned kPlaneBytes3 = kPlane3 * 4u;

size_t step3d_smem_bytes() { return (size_t)kRing * kPlaneBytes3 + (size_t)kTY3 * kTX * 4; }

__device__ __forceinline__ float sponge_e3(const ModelStep3D& M, int z, int y, int x) {
    const int rz = max(max(M.pad - z, z - (M.pad + M.nz - 1)), 0);
    const int ry = max(max(M.pad - y, y - (M.pad + M.ny - 1)), 0);
    const int rx = max(max(M.pad - x, x - (M.pad + M.nx - 1)), 0);
    return __fmaf_rn(M.cz, (float)(rz * rz), __fmaf_rn(M.cy, (float)(ry * ry), __fmul_rn(M.cx, (float)(rx * rx))));
}

template <int MODE, bool KAHAN>
__global__ void __launch_bounds__(kThreads) k_step3d(const __grid_constant__ StepParams3D p) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[kRing];
    const ModelStep3D& M = p.m;
    const int tid = threadIdx.x;
    const int lx = (tid & 15) << 2, ly = tid >> 4;
    int t = blockIdx.x;
    const int txi = t % M.tiles_x;
    t /= M.tiles_x;
    const int tyi = t % M.tiles_y;
    const int zc = t / M.tiles_y;
    const int x0 = txi * kTX, y0 = tyi * kTY3, z0 = zc * M.ZC;
    const int zend = min(z0 + M.ZC, M.Nz);
    const int fidx = blockIdx.y;  // shot * nfield + field
    const int shot = fidx / M.nfield;
    const int b = fidx - shot * M.nfield;
    const int n = p.n;
    const int pc = (MODE == STEP3_ADJ) ? ((n + 1) & 1) : (n & 1);
    const int po = pc ^ 1;
    const long long F = M.F;
    const int vol_cur = shot * M.nvol_shot + 2 * b + pc;
    float* outv = M.state + (long long)(shot * M.nvol_shot + 2 * b + po) * F;
    float* sinj = smem + kRing * kPlane3;
    const int nplanes = (zend - z0) + 8;

    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < min(kRing, nplanes); ++k) {
            mbar_expect_tx(&bars[k], kPlaneBytes3);
            tma_load_4d(smem + k * kPlane3, &M.tm, x0 - 4, y0 - 4, z0 - 4 + k, vol_cur, &bars[k]);
        }
    }

    const int x = x0 + lx, y = y0 + ly;
    const bool col_ok = (x < M.Nx) && (y < M.Ny);
    const bool interior_col = (x >= M.pad) && (x + 3 < M.pad + M.nx) && (y >= M.pad) && (y < M.pad + M.ny);
    const int sz = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.src[3 * shot] : -1;
    const int sy = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.src[3 * shot + 1] : -1;
    const int sx = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.src[3 * shot + 2] : -1;
    const float fsrc = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.wavelet[n] * M.vol_inv : 0.f;
    const int tile_xy = tyi * M.tiles_x + txi;

    for (int iz = 0; iz < zend - z0; ++iz) {
        const int z = z0 + iz;
        // all planes up to k = iz + 8 must have landed
        const int kfirst = (iz == 0) ? 0 : iz + 8;
        for (int k = kfirst; k <= iz + 8; ++k) {
            const bool ok = mbar_wait_bounded(&bars[k % kRing], (uint32_t)((k / kRing) & 1));
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    // flag the error, then give the copies still in flight one more bounded wait
                    set_dev_error(p.err, DEVERR_TIMEOUT);
                    const int issued = min(nplanes, iz - 1 + kRing + 1);
                    for (int q = k; q < issued; ++q)
                        (void)mbar_wait_bounded(&bars[q % kRing], (uint32_t)((q / kRing) & 1));
                }
                return;
            }
        }
        // receivers of this plane (Born sampling / adjoint injection)
        const int rk = tile_xy * M.Nz + z;
        const int rbeg = M.rec_ptr[rk], rend = M.rec_ptr[rk + 1];
        const float* cur = smem + ((iz + 4) % kRing) * kPlane3;
        if (MODE == STEP3_BORN || MODE == STEP3_INC_SAMPLE) {
            if (rend > rbeg) {
                float* dout = M.data + (long long)shot * M.dss + (long long)b * M.dts + (long long)n * M.nr;
                for (int i = rbeg + tid; i < rend; i += kThreads) {
                    const int r = M.rec_idx[i];
                    dout[r] = cur[(M.rec_zyx[3 * r + 1] - y0 + 4) * kHX3 + (M.rec_zyx[3 * r + 2] - x0 + 4)];
                }
            }
        }
        const bool inj = (MODE == STEP3_ADJ) && (rend > rbeg);
        if (inj) {
            for (int i = tid; i < kTY3 * kTX; i += kThreads) sinj[i] = 0.f;
            __syncthreads();
            const float* rr = M.rdata + (long long)shot * M.dss + (long long)b * M.dts + (long long)n * M.nr;
            for (int i = rbeg + tid; i < rend; i += kThreads) {
                const int r = M.rec_idx[i];
                atomicAdd(&sinj[(M.rec_zyx[3 * r + 1] - y0) * kTX + (M.rec_zyx[3 * r + 2] - x0)], rr[r]);
            }
            __syncthreads();
        }
        if (col_ok && z < M.Nz) {
            const long long off = ((long long)z * M.Ny + y) * M.P + x;
            const float* rp = cur + (ly + 4) * kHX3 + lx + 4;
            const float4 a = ld4(rp - 4), c = ld4(rp), d = ld4(rp + 4);
            const float v[12] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
            float L[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float u0 = v[4 + j];
                float acc = 0.f;
#pragma unroll
                for (int k = 1; k <= 4; ++k) acc = fmaf(M.lx[k - 1], (v[4 + j + k] - u0) + (v[4 + j - k] - u0), acc);
                L[j] = acc;
            }
#pragma unroll
            for (int k = 1; k <= 4; ++k) {
                const float4 up = ld4(rp - k * kHX3), dn = ld4(rp + k * kHX3);
                const float w = M.ly[k - 1];
                L[0] = fmaf(w, (up.x - c.x) + (dn.x - c.x), L[0]);
                L[1] = fmaf(w, (up.y - c.y) + (dn.y - c.y), L[1]);
                L[2] = fmaf(w, (up.z - c.z) + (dn.z - c.z), L[2]);
                L[3] = fmaf(w, (up.w - c.w) + (dn.w - c.w), L[3]);
            }
#pragma unroll
            for (int k = 1; k <= 4; ++k) {
                const float4 up = ld4(smem + ((iz + 4 - k) % kRing) * kPlane3 + (ly + 4) * kHX3 + lx + 4);
                const float4 dn = ld4(smem + ((iz + 4 + k) % kRing) * kPlane3 + (ly + 4) * kHX3 + lx + 4);
                const float w = M.lz[k - 1];
                L[0] = fmaf(w, (up.x - c.x) + (dn.x - c.x), L[0]);
                L[1] = fmaf(w, (up.y - c.y) + (dn.y - c.y), L[1]);
                L[2] = fmaf(w, (up.z - c.z) + (dn.z - c.z), L[2]);
                L[3] = fmaf(w, (up.w - c.w) + (dn.w - c.w), L[3]);
            }
            const float4 sv = ld4(M.s + off);
            const float4 ov = ld4(outv + off);
            float src[4] = {0.f, 0.f, 0.f, 0.f};
            float Dv[4] = {0.f, 0.f, 0.f, 0.f};
            if (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) {
                if (z == sz && y == sy) {
                    const int j = sx - x;
                    add_lane(src, j, fsrc);
                }
            } else if (MODE == STEP3_BORN) {
                const float4 dd = ld4(M.Din + (long long)shot * M.Din_shot_stride + off);
                const float4 dmv = ld4(M.dm + (long long)b * F + off);
                L[0] = __fmaf_rn(-dmv.x, dd.x, L[0]);  // Born source -dm Dtt u folded into L
                L[1] = __fmaf_rn(-dmv.y, dd.y, L[1]);
                L[2] = __fmaf_rn(-dmv.z, dd.z, L[2]);
                L[3] = __fmaf_rn(-dmv.w, dd.w, L[3]);
            } else {
                const float4 dd = ld4(M.Din + (long long)shot * M.Din_shot_stride + off);
                Dv[0] = dd.x;
                Dv[1] = dd.y;
                Dv[2] = dd.z;
                Dv[3] = dd.w;
                if (inj) {
                    const float4 iv = ld4(sinj + ly * kTX + lx);
                    src[0] = iv.x;
                    src[1] = iv.y;
                    src[2] = iv.z;
                    src[3] = iv.w;
                }
            }
            const bool interior = interior_col && (z >= M.pad) && (z < M.pad + M.nz);
            float o[4], Dw[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float G = 1.f, am = 1.f;
                if (!interior) sponge_pair(sponge_e3(M, z, y, x + j), G, am);
                const float Fo = __fmul_rn(get(sv, j), __fadd_rn(L[j], src[j]));
                Dw[j] = __fmul_rn(Fo, M.inv_dt2);
                o[j] = (x + j < M.Nx) ? leapfrog(G, v[4 + j], am, get(ov, j), Fo) : 0.f;
            }
            st4(outv + off, make_float4(o[0], o[1], o[2], o[3]));
            if ((MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) && M.Dout)
                st4(M.Dout + (long long)shot * M.Dout_shot_stride + off, make_float4(Dw[0], Dw[1], Dw[2], Dw[3]));
            if (MODE == STEP3_ADJ) {
                float* ip = M.img + (long long)(shot * M.nfield + b) * F + off;
                float4 iv = ld4(ip);
                const float t0 = __fmul_rn(-Dv[0], o[0]), t1 = __fmul_rn(-Dv[1], o[1]);
                const float t2 = __fmul_rn(-Dv[2], o[2]), t3 = __fmul_rn(-Dv[3], o[3]);
                if (KAHAN) {
                    float* cp = M.comp + (long long)(shot * M.nfield + b) * F + off;
                    float4 cv = ld4(cp);
                    kahan4(iv, cv, t0, t1, t2, t3);
                    st4(cp, cv);
                } else {
                    iv.x = __fadd_rn(iv.x, t0);
                    iv.y = __fadd_rn(iv.y, t1);
                    iv.z = __fadd_rn(iv.z, t2);
                    iv.w = __fadd_rn(iv.w, t3);
                }
                st4(ip, iv);
            }
        }
        __syncthreads();  // the slot of plane k = iz is free again
        if (tid == 0) {
            const int k = iz + kRing;
            if (k < nplanes) {
                mbar_expect_tx(&bars[k % kRing], kPlaneBytes3);
                tma_load_4d(smem + (k % kRing) * kPlane3, &M.tm, x0 - 4, y0 - 4, z0 - 4 + k, vol_cur,
                            &bars[k % kRing]);
            }
        }
    }
}

template <int MODE, bool KAHAN>
static cudaError_t launch3(const StepParams3D& p, dim3 grid, cudaStream_t st) {
    const size_t sm = step3d_smem_bytes();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_step3d<MODE, KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_step3d<MODE, KAHAN><<<grid, kThreads, sm, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_step3d(int mode, bool kahan, const StepParams3D& p, cudaStream_t st) {
    const ModelStep3D& M = p.m;
    dim3 grid(M.tiles_x * M.tiles_y * M.zchunks, M.nshots * M.nfield);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    switch (mode) {
        case STEP3_INC: return launch3<STEP3_INC, false>(p, grid, st);
        case STEP3_INC_SAMPLE: return launch3<STEP3_INC_SAMPLE, false>(p, grid, st);
        case STEP3_BORN: return launch3<STEP3_BORN, false>(p, grid, st);
        case STEP3_ADJ:
            return kahan ? launch3<STEP3_ADJ, true>(p, grid, st) : launch3<STEP3_ADJ, false>(p, grid, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace probe
