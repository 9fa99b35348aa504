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
constexpr int kPrefetch3 = 2;   // planes ahead whose pointwise operands are prefetched into L2
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

// Sponge factors G, a- of a thread's 4 cells on the planes where z is not in the sponge: there
// the exponent has no z part, so they depend on the column alone and are formed once per CTA
// (1 on interior columns).  Same roundings as sponge_pair(sponge_e3(...)) on those planes.
__device__ __forceinline__ void sponge_col3(const ModelStep3D& M, int y, int x, float4& G, float4& A) {
    float g[4], a[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        g[j] = 1.f;
        a[j] = 1.f;
        sponge_pair(sponge_e3(M, M.pad, y, x + j), g[j], a[j]);
    }
    G = make_float4(g[0], g[1], g[2], g[3]);
    A = make_float4(a[0], a[1], a[2], a[3]);
}

// Pointwise operands of one plane of a thread's 4 cells, loaded at the top of that plane (after an
// L2 prefetch kPrefetch3 planes earlier) so that their latency overlaps the ring wait and the taps.
struct Pw3 {
    float4 s, prev, d, dm, img, cmp;
};

template <int MODE, bool KAHAN>
__device__ __forceinline__ void load_pw3(const ModelStep3D& M, const float* outv, long long off, int shot, int b,
                                         long long F, Pw3& w) {
    w.s = ld4(M.s + off);
    w.prev = ld4(outv + off);
    if (MODE == STEP3_BORN || MODE == STEP3_ADJ) w.d = ld4(M.Din + (long long)shot * M.Din_shot_stride + off);
    if (MODE == STEP3_BORN) w.dm = ld4(M.dm + (long long)b * F + off);
    if (MODE == STEP3_ADJ) {
        if (!M.seg_first) w.img = ld4(M.img + (long long)(shot * M.nfield + b) * F + off);
        if (KAHAN) w.cmp = ld4(M.comp + (long long)(shot * M.nfield + b) * F + off);
    }
}

// The same operands two planes ahead, brought into L2 only (no registers held).
template <int MODE, bool KAHAN>
__device__ __forceinline__ void prefetch_pw3(const ModelStep3D& M, const float* outv, long long off, int shot, int b,
                                             long long F) {
    prefetch_l2(M.s + off);
    prefetch_l2(outv + off);
    if (MODE == STEP3_BORN || MODE == STEP3_ADJ) prefetch_l2(M.Din + (long long)shot * M.Din_shot_stride + off);
    if (MODE == STEP3_BORN) prefetch_l2(M.dm + (long long)b * F + off);
    if (MODE == STEP3_ADJ) {
        if (!M.seg_first) prefetch_l2(M.img + (long long)(shot * M.nfield + b) * F + off);
        if (KAHAN) prefetch_l2(M.comp + (long long)(shot * M.nfield + b) * F + off);
    }
}

// Update of one z plane of a thread's 4 cells, once every plane the taps need is in the ring:
// slot_c holds the current plane (halo tile), slot_c -+ k the planes k below / above; cur_pw
// the cells' pointwise operands; injv the receiver injection of the cells (adjoint, when inj).
template <int MODE, bool KAHAN>
__device__ __forceinline__ void cells3(const ModelStep3D& M, const float* smem, int slot_c, int lx, int ly, int x,
                                       int y, int z, long long off, int shot, int b, long long F, float* outv,
                                       const Pw3& cur_pw, const float4& Gc, const float4& Ac, int sz, int sy,
                                       int sx, float fsrc, bool inj, float4 injv,
                                       float4* dtt_out = nullptr, float4* prod_out = nullptr,
                                       const float* injq = nullptr) {
    const float* cur = smem + slot_c * kPlane3;
    const float* rp = cur + (ly + 4) * kHX3 + lx + 4;
    const float4 a = ld4(rp - 4), c = ld4(rp), d = ld4(rp + 4);
    // x taps in first-difference form (11 shared differences for the 4 cells)
    const float v[12] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
    float dx[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) dx[i] = v[i + 1] - v[i];
    float L[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float acc = M.cxm[0] * (dx[4 + j] - dx[3 + j]);
#pragma unroll
        for (int m = 1; m < 4; ++m) acc = fmaf(M.cxm[m], dx[4 + j + m] - dx[3 + j - m], acc);
        L[j] = acc;
    }
    // y and z taps, (v_{+k} - c) + (v_{-k} - c) per pair, in packed FP32x2 (same roundings per lane)
    P4 acc = p4(L[0], L[1], L[2], L[3]);
    const P4 cc = p4(c);
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        const P4 up = p4(ld4(rp - k * kHX3)), dn = p4(ld4(rp + k * kHX3));
        const float w = M.ly[k - 1];
        acc = p4fma(p4(w, w, w, w), p4add(p4sub(up, cc), p4sub(dn, cc)), acc);
    }
    const int cofs = (ly + 4) * kHX3 + lx + 4;
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        int su = slot_c - k, sd = slot_c + k;
        su += (su < 0) ? kRing : 0;
        sd -= (sd >= kRing) ? kRing : 0;
        const P4 up = p4(ld4(smem + su * kPlane3 + cofs));
        const P4 dn = p4(ld4(smem + sd * kPlane3 + cofs));
        const float w = M.lz[k - 1];
        acc = p4fma(p4(w, w, w, w), p4add(p4sub(up, cc), p4sub(dn, cc)), acc);
    }
    {
        const float4 a4 = f4(acc);
        L[0] = a4.x;
        L[1] = a4.y;
        L[2] = a4.z;
        L[3] = a4.w;
    }
    const float4 sv = cur_pw.s;
    const float4 ov = cur_pw.prev;
    float src[4] = {0.f, 0.f, 0.f, 0.f};
    float Dv[4] = {0.f, 0.f, 0.f, 0.f};
    if (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) {
        if (z == sz && y == sy) add_lane(src, sx - x, fsrc);
    } else if (MODE == STEP3_BORN) {
        const float4 dd = cur_pw.d;
        const float4 dmv = cur_pw.dm;
        L[0] = __fmaf_rn(-dmv.x, dd.x, L[0]);  // Born source -dm Dtt u folded into L
        L[1] = __fmaf_rn(-dmv.y, dd.y, L[1]);
        L[2] = __fmaf_rn(-dmv.z, dd.z, L[2]);
        L[3] = __fmaf_rn(-dmv.w, dd.w, L[3]);
    } else {
        const float4 dd = cur_pw.d;
        Dv[0] = dd.x;
        Dv[1] = dd.y;
        Dv[2] = dd.z;
        Dv[3] = dd.w;
        if (inj) {
            src[0] = injv.x;
            src[1] = injv.y;
            src[2] = injv.z;
            src[3] = injv.w;
        } else if (injq) {  // injection read at its use (receiver planes only: no register held over the taps)
            const float4 q = ld4(injq);
            src[0] = q.x;
            src[1] = q.y;
            src[2] = q.z;
            src[3] = q.w;
        }
    }
    const bool zin = (z >= M.pad) && (z < M.pad + M.nz);
    float o[4], Dw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float G = get(Gc, j), am = get(Ac, j);  // planes outside the z sponge: the column's factors
        if (!zin) {
            G = 1.f;
            am = 1.f;
            sponge_pair(sponge_e3(M, z, y, x + j), G, am);
        }
        const float Fo = __fmul_rn(get(sv, j), __fadd_rn(L[j], src[j]));
        Dw[j] = __fmul_rn(Fo, M.inv_dt2);
        o[j] = (x + j < M.Nx) ? leapfrog(G, v[4 + j], am, get(ov, j), Fo) : 0.f;
    }
    st4(outv + off, make_float4(o[0], o[1], o[2], o[3]));
    if ((MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) && M.Dout)
        st4(M.Dout + (long long)shot * M.Dout_shot_stride + off, make_float4(Dw[0], Dw[1], Dw[2], Dw[3]));
    if ((MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) && dtt_out) *dtt_out = make_float4(Dw[0], Dw[1], Dw[2], Dw[3]);
    if (MODE == STEP3_ADJ) {
        const float t0 = __fmul_rn(-Dv[0], o[0]), t1 = __fmul_rn(-Dv[1], o[1]);
        const float t2 = __fmul_rn(-Dv[2], o[2]), t3 = __fmul_rn(-Dv[3], o[3]);
        if (prod_out) {  // the caller accumulates the image (shot-cluster kernel)
            *prod_out = make_float4(t0, t1, t2, t3);
            return;
        }
        float* ip = M.img + (long long)(shot * M.nfield + b) * F + off;
        float4 iv = cur_pw.img;
        if (KAHAN) {
            float* cp = M.comp + (long long)(shot * M.nfield + b) * F + off;
            float4 cv = cur_pw.cmp;
            kahan4(iv, cv, t0, t1, t2, t3);
            st4(cp, cv);
        } else if (M.seg_first) {
            iv = make_float4(t0, t1, t2, t3);
        } else {
            iv.x = __fadd_rn(iv.x, t0);
            iv.y = __fadd_rn(iv.y, t1);
            iv.z = __fadd_rn(iv.z, t2);
            iv.w = __fadd_rn(iv.w, t3);
        }
        st4(ip, iv);
    }
}

template <int MODE, bool KAHAN>
__global__ void __launch_bounds__(kThreads, 3) k_step3d(const __grid_constant__ StepParams3D p) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[kRing];
    constexpr bool RECV = (MODE != STEP3_INC);  // receivers: sampling (Born, nonlinear) or injection (adjoint)
    const ModelStep3D& M = p.m;
    const int tid = threadIdx.x;
    const int lx = (tid & 15) << 2, ly = tid >> 4;
    // grid.x = (column tile, chunk) x field with the field fastest: the fields of one tile run as
    // neighbouring CTAs, so the operands they share (s, a shot's Dtt) come from L2 after the first
    const int b = (int)(blockIdx.x % M.nfield);
    int t = (int)(blockIdx.x / M.nfield);
    const int txi = t % M.tiles_x;
    t /= M.tiles_x;
    const int tyi = t % M.tiles_y;
    const int zc = t / M.tiles_y;
    const int x0 = txi * kTX, y0 = tyi * kTY3, z0 = zc * M.ZC;
    const int zend = min(z0 + M.ZC, M.Nz);
    const int shot = blockIdx.y;
    const int n = p.n;
    const int pc = (MODE == STEP3_ADJ) ? ((n + 1) & 1) : (n & 1);
    const int po = pc ^ 1;
    const long long F = M.F;
    const int vol_cur = shot * M.nvol_shot + 2 * b + pc;
    float* outv = M.state + (long long)(shot * M.nvol_shot + 2 * b + po) * F;
    float* sinj = smem + kRing * kPlane3;
    const int nloc = zend - z0;
    const int nplanes = nloc + 8;

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
    float4 Gc, Ac;
    sponge_col3(M, y, x, Gc, Ac);
    const int sz = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.src[3 * shot] : -1;
    const int sy = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.src[3 * shot + 1] : -1;
    const int sx = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.src[3 * shot + 2] : -1;
    const float fsrc = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.wavelet[n] * M.vol_inv : 0.f;
    const int tile_xy = tyi * M.tiles_x + txi;
    const long long plane_stride = (long long)M.Ny * M.P;
    const long long off0 = ((long long)z0 * M.Ny + y) * M.P + x;

    // ring bookkeeping without divisions: slot of the current plane (k = iz + 4) and of the
    // farthest plane the taps need (k = iz + 8), with that slot's mbarrier phase
    int slot_c = 4, slot_w = 8;
    uint32_t ph_w = 0;

    // one z plane; the operands of this plane arrived in cur_pw, the next plane's go to nxt_pw
    auto plane = [&](int iz) -> bool {
        const int z = z0 + iz;
        Pw3 cur_pw;  // this plane's operands, in flight during the ring wait and the stencil
        if (col_ok) load_pw3<MODE, KAHAN>(M, outv, off0 + (long long)iz * plane_stride, shot, b, F, cur_pw);
        if (col_ok && iz + kPrefetch3 < nloc)
            prefetch_pw3<MODE, KAHAN>(M, outv, off0 + (long long)(iz + kPrefetch3) * plane_stride, shot, b, F);
        // every plane up to k = iz + 8 must have landed
        const int kfirst = (iz == 0) ? 0 : iz + 8;
        for (int k = kfirst; k <= iz + 8; ++k) {
            const bool ok = (iz == 0) ? mbar_wait_bounded(&bars[k], 0u) : mbar_wait_bounded(&bars[slot_w], ph_w);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    // flag the error, then give the copies still in flight one more bounded wait
                    set_dev_error(p.err, DEVERR_TIMEOUT);
                    const int issued = min(nplanes, iz + kRing);
                    for (int q = k; q < issued; ++q)
                        (void)mbar_wait_bounded(&bars[q % kRing], (uint32_t)((q / kRing) & 1));
                }
                return false;
            }
        }
        const float* cur = smem + slot_c * kPlane3;
        int rbeg = 0, rend = 0;
        if (RECV) {  // receivers of this plane (Born / nonlinear sampling, adjoint injection)
            const int rk = tile_xy * M.Nz + z;
            rbeg = M.rec_ptr[rk];
            rend = M.rec_ptr[rk + 1];
        }
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
        if (col_ok && z < M.Nz)
            cells3<MODE, KAHAN>(M, smem, slot_c, lx, ly, x, y, z, off0 + (long long)iz * plane_stride, shot, b, F, outv,
                                cur_pw, Gc, Ac, sz, sy, sx, fsrc, inj,
                                inj ? ld4(sinj + ly * kTX + lx) : make_float4(0.f, 0.f, 0.f, 0.f));
        __syncthreads();  // the slot of plane k = iz is free again
        if (tid == 0) {
            const int k = iz + kRing;
            if (k < nplanes) {
                int sf = slot_c - 4;  // slot of plane iz
                sf += (sf < 0) ? kRing : 0;
                mbar_expect_tx(&bars[sf], kPlaneBytes3);
                tma_load_4d(smem + sf * kPlane3, &M.tm, x0 - 4, y0 - 4, z0 - 4 + k, vol_cur, &bars[sf]);
            }
        }
        slot_c = (slot_c + 1 == kRing) ? 0 : slot_c + 1;
        if (++slot_w == kRing) {
            slot_w = 0;
            ph_w ^= 1u;
        }
        return true;
    };

    // unrolled by two: the next plane's loads can then be scheduled into this plane's work
#pragma unroll 2
    for (int iz = 0; iz < nloc; ++iz)
        if (!plane(iz)) return;
}

constexpr int kWs3Threads = kThreads + 32;  // eight consumer warps + one producer warp

// Pipelined variant (incident, nonlinear sampling, Born, and the adjoint without per-step Kahan
// compensation): the halo'd planes stream into the ring against per-slot full mbarriers, and the
// compute warps never meet at a CTA-wide barrier inside the plane loop; each releases the oldest
// plane of its window as soon as it is done with it.  With PROD, one producer warp waits on
// per-slot empty mbarriers (one arrival per compute warp) and issues the refills; without it,
// each compute warp counts itself out of the slot on a shared counter and the last of the eight
// issues the slot's next TMA load itself, so no warp polls for free slots and the CTA is eight
// warps, which leaves the compute warps more registers at three CTAs per SM.  The adjoint's receiver injection R^T r^n comes from the
// segment's prebuilt band buffer (one float4 per thread on the planes that hold receivers)
// instead of being assembled in shared memory.  The per-cell arithmetic is cells3, identical to
// k_step3d.  Every wait is bounded.
template <int MODE, bool PROD>
__global__ void __launch_bounds__(PROD ? kWs3Threads : kThreads, 3) k_step3d_ws(const __grid_constant__ StepParams3D p) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t full[kRing], empty[kRing];
    __shared__ uint32_t released[kRing];  // without PROD: compute-warp releases of each slot, cumulative
    // receiver CSR bounds of this column tile's planes (sampling), or each plane's injection
    // band, -1 without receivers (adjoint)
    __shared__ int srec[kZCMax3D + 1];
    constexpr bool SAMPLE = (MODE == STEP3_BORN || MODE == STEP3_INC_SAMPLE);
    constexpr bool ADJ = (MODE == STEP3_ADJ);
    const ModelStep3D& M = p.m;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // grid.x = (column tile, chunk) x field with the field fastest: the fields of one tile run as
    // neighbouring CTAs, so the operands they share (s, a shot's Dtt) come from L2 after the first
    const int b = (int)(blockIdx.x % M.nfield);
    int t = (int)(blockIdx.x / M.nfield);
    const int txi = t % M.tiles_x;
    t /= M.tiles_x;
    const int tyi = t % M.tiles_y;
    const int zc = t / M.tiles_y;
    const int x0 = txi * kTX, y0 = tyi * kTY3, z0 = zc * M.ZC;
    const int zend = min(z0 + M.ZC, M.Nz);
    const int shot = blockIdx.y;
    const int n = p.n;
    const int pc = ADJ ? ((n + 1) & 1) : (n & 1), po = pc ^ 1;
    const long long F = M.F;
    const int vol_cur = shot * M.nvol_shot + 2 * b + pc;
    float* outv = M.state + (long long)(shot * M.nvol_shot + 2 * b + po) * F;
    const int nloc = zend - z0;
    const int nplanes = nloc + 8;

    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kThreads / 32);
            released[i] = 0u;
        }
        fence_mbar_init();
    }
    if (SAMPLE && tid <= nloc) srec[tid] = M.rec_ptr[(tyi * M.tiles_x + txi) * M.Nz + z0 + tid];
    if (ADJ && tid < nloc) srec[tid] = (M.rrow && M.inj) ? M.rrow[z0 + tid] : -1;
    __syncthreads();
    if (!PROD && tid == 0) {  // the first kRing planes; the compute warps issue the rest
        for (int k = 0; k < min(kRing, nplanes); ++k) {
            mbar_expect_tx(&full[k], kPlaneBytes3);
            tma_load_4d(smem + k * kPlane3, &M.tm, x0 - 4, y0 - 4, z0 - 4 + k, vol_cur, &full[k]);
        }
    }

    if (PROD && warp == kThreads / 32) {  // ---------------- producer warp
        if (lane != 0) return;
        int sl = 0;
        uint32_t eph = 0;  // phase of empty[sl] to wait for, once the ring has wrapped
        for (int k = 0; k < nplanes; ++k) {
            if (k >= kRing && !mbar_wait_bounded(&empty[sl], eph)) {
                set_dev_error(p.err, DEVERR_TIMEOUT);
                return;
            }
            mbar_expect_tx(&full[sl], kPlaneBytes3);
            tma_load_4d(smem + sl * kPlane3, &M.tm, x0 - 4, y0 - 4, z0 - 4 + k, vol_cur, &full[sl]);
            if (++sl == kRing) {
                sl = 0;
                if (k + 1 >= 2 * kRing) eph ^= 1u;  // the wait for plane k + 1 is for its (k+1)/kRing - 1 th release
            }
        }
        return;
    }

    // ---------------- consumer warps
    const int lx = (tid & 15) << 2, ly = tid >> 4;
    const int x = x0 + lx, y = y0 + ly;
    const bool col_ok = (x < M.Nx) && (y < M.Ny);
    float4 Gc, Ac;
    sponge_col3(M, y, x, Gc, Ac);
    const int sz = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.src[3 * shot] : -1;
    const int sy = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.src[3 * shot + 1] : -1;
    const int sx = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.src[3 * shot + 2] : -1;
    const float fsrc = (MODE == STEP3_INC || MODE == STEP3_INC_SAMPLE) ? M.wavelet[n] * M.vol_inv : 0.f;
    const long long plane_stride = (long long)M.Ny * M.P;
    const long long off0 = ((long long)z0 * M.Ny + y) * M.P + x;
    int slot_c = 4, slot_w = 8;  // slots of the current plane (k = iz + 4) and of k = iz + 8
    uint32_t ph_w = 0;

    auto plane = [&](int iz) -> bool {
        const int z = z0 + iz;
        // this plane's pointwise operands (prefetched into L2 earlier): issued before the ring
        // wait so that their latency overlaps the wait and the stencil
        Pw3 cur_pw;
        if (col_ok) load_pw3<MODE, false>(M, outv, off0 + (long long)iz * plane_stride, shot, b, F, cur_pw);
        if (col_ok && iz + kPrefetch3 < nloc)
            prefetch_pw3<MODE, false>(M, outv, off0 + (long long)(iz + kPrefetch3) * plane_stride, shot, b, F);
        const int kfirst = (iz == 0) ? 0 : iz + 8;
        for (int k = kfirst; k <= iz + 8; ++k) {
            const bool ok = (iz == 0) ? mbar_wait_bounded(&full[k], 0u) : mbar_wait_bounded(&full[slot_w], ph_w);
            if (!ok) {
                set_dev_error(p.err, DEVERR_TIMEOUT);
                return false;
            }
        }
        if (SAMPLE) {  // receivers of this plane, from its staged tile
            const int rbeg = srec[iz], rend = srec[iz + 1];
            if (rend > rbeg) {
                const float* cur = smem + slot_c * kPlane3;
                float* dout = M.data + (long long)shot * M.dss + (long long)b * M.dts + (long long)n * M.nr;
                for (int i = rbeg + tid; i < rend; i += kThreads) {
                    const int r = M.rec_idx[i];
                    dout[r] = cur[(M.rec_zyx[3 * r + 1] - y0 + 4) * kHX3 + (M.rec_zyx[3 * r + 2] - x0 + 4)];
                }
            }
        }
        // the receiver injection of this plane's cells (adjoint): band srec[iz] of the segment's
        // buffer, one Ny x P plane per band
        const float* injq = nullptr;
        if (ADJ && srec[iz] >= 0)
            injq = M.inj + ((long long)(M.inj_slot * M.nshots + shot) * M.nfield + b) * M.inj_block +
                   (long long)srec[iz] * plane_stride + (long long)y * M.P + x;
        if (col_ok && z < M.Nz)
            cells3<MODE, false>(M, smem, slot_c, lx, ly, x, y, z, off0 + (long long)iz * plane_stride, shot, b, F,
                                outv, cur_pw, Gc, Ac, sz, sy, sx, fsrc, false, make_float4(0.f, 0.f, 0.f, 0.f),
                                nullptr, nullptr, injq);
        __syncwarp();
        if (lane == 0) {  // this warp is done with plane k = iz (the bottom of its window)
            int sf = slot_c - 4;
            sf += (sf < 0) ? kRing : 0;
            if (PROD) {
                mbar_arrive(&empty[sf]);
            } else {
                // the slot's use u = iz / kRing ends with the (8u + 8)-th release: that warp
                // refills the slot with ring plane iz + kRing
                const uint32_t old = atom_add_acqrel_shared(&released[sf], 1u);
                const uint32_t last = (uint32_t)(kThreads / 32) * (uint32_t)(iz / kRing + 1) - 1u;
                const int k = iz + kRing;
                if (old == last && k < nplanes) {
                    fence_proxy_async_shared();
                    mbar_expect_tx(&full[sf], kPlaneBytes3);
                    tma_load_4d(smem + sf * kPlane3, &M.tm, x0 - 4, y0 - 4, z0 - 4 + k, vol_cur, &full[sf]);
                }
            }
        }
        slot_c = (slot_c + 1 == kRing) ? 0 : slot_c + 1;
        if (++slot_w == kRing) {
            slot_w = 0;
            ph_w ^= 1u;
        }
        return true;
    };

    if (ADJ) {  // one plane per iteration: fewer registers spilled with the adjoint's operands
#pragma unroll 1
        for (int iz = 0; iz < nloc; ++iz)
            if (!plane(iz)) return;
    } else {
#pragma unroll 2
        for (int iz = 0; iz < nloc; ++iz)
            if (!plane(iz)) return;
    }
}

// ---------------------------------------------------------------------------------------------
// Fused forward step (incident + Born trials) on a thread-block cluster.
//
// The cluster of one column tile and one shot holds 1 + nb CTAs: rank 0 advances the incident
// field u0, rank 1 + b the Born field of trial b.  Each CTA streams its own field's halo'd planes
// through its TMA ring (producer warp, per-slot full / empty mbarriers, as k_step3d_ws).  The
// Born source needs Dtt u0^n of the same cells: rank 0 computes it in registers while updating
// u0 and stores it straight into a small ring of Dtt planes in every Born CTA's shared memory
// (distributed shared memory), then arrives on that slot's mbarrier in each of them; a Born CTA
// releases the slot by arriving on rank 0's matching mbarrier.  Dtt u0 therefore never goes to
// HBM: per cell and step the fused step moves u0^n, u0^{n-1}, s, u0^{n+1} and, per trial, du^n,
// du^{n-1}, dm, du^{n+1} -- (16 + 16 nb) bytes instead of the 20 + 24 nb of separate incident
// and Born launches.  The per-cell arithmetic is cells3, so the results are the same bits as
// the separate launches.  Every wait is bounded; a CTA that gives up leaves its plane loop and
// still meets the closing cluster barrier, so no CTA leaves while another can reach its shared
// memory.
// ---------------------------------------------------------------------------------------------
constexpr int kDslots = 4;                 // Dtt planes in flight from rank 0 to the Born CTAs
constexpr int kTile3 = kTY3 * kTX;          // cells of a column tile's plane
constexpr int kMaxCluster3 = 8;             // portable cluster size: 1 + nb <= 8

size_t fwd3d_cluster_smem_bytes() { return (size_t)kRing * kPlaneBytes3 + (size_t)kDslots * kTile3 * 4; }

__global__ void __launch_bounds__(kWs3Threads, 2) k_fwd3d_cl(const __grid_constant__ StepParams3D p) {
    extern __shared__ __align__(128) float smem[];  // [kRing][kPlane3] ring, then [kDslots][kTile3] Dtt
    __shared__ __align__(8) uint64_t full[kRing], empty[kRing], dfull[kDslots], dempty[kDslots];
    __shared__ int srec[kZCMax3D + 1];
    const int nb = p.m2.nfield;
    const int nf = nb + 1;
    const uint32_t rank = cluster_ctarank();  // == blockIdx.x % nf: the field of this CTA
    const bool inc = (rank == 0);
    const ModelStep3D& M = inc ? p.m : p.m2;
    const int b = inc ? 0 : (int)rank - 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int t = (int)(blockIdx.x / nf);
    const int txi = t % M.tiles_x;
    t /= M.tiles_x;
    const int tyi = t % M.tiles_y;
    const int zc = t / M.tiles_y;
    const int x0 = txi * kTX, y0 = tyi * kTY3, z0 = zc * M.ZC;
    const int zend = min(z0 + M.ZC, M.Nz);
    const int shot = blockIdx.y;
    const int n = p.n;
    const int pc = n & 1, po = pc ^ 1;
    const long long F = M.F;
    const int vol_cur = shot * M.nvol_shot + 2 * b + pc;
    float* outv = M.state + (long long)(shot * M.nvol_shot + 2 * b + po) * F;
    const int nloc = zend - z0;
    const int nplanes = nloc + 8;
    float* dslots = smem + kRing * kPlane3;

    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kThreads / 32);
        }
        for (int i = 0; i < kDslots; ++i) {
            mbar_init(&dfull[i], 1);                      // armed for one plane of asynchronous stores
            mbar_init(&dempty[i], (kThreads / 32) * nb);  // every Born CTA's consumer warps
        }
        if (!inc)
            for (int i = 0; i < kDslots; ++i) mbar_arm_tx(&dfull[i], kTile3 * 4);
        fence_mbar_init();
    }
    if (!inc && tid <= nloc) srec[tid] = M.rec_ptr[(tyi * M.tiles_x + txi) * M.Nz + z0 + tid];
    __syncthreads();
    cluster_sync_all();  // all barriers of the cluster exist before the first remote arrival
    // after an earlier failure (a wait that gave up) the remaining CTAs do no work
    const bool skip = *reinterpret_cast<volatile int*>(p.err) != 0;

    if (warp == kThreads / 32) {  // ---------------- producer warp
        if (lane == 0 && !skip) {
            int sl = 0, issued = 0;
            uint32_t eph = 0;
            for (int k = 0; k < nplanes; ++k) {
                if (k >= kRing && !mbar_wait_bounded(&empty[sl], eph)) {
                    set_dev_error(p.err, DEVERR_TIMEOUT);
                    break;
                }
                mbar_expect_tx(&full[sl], kPlaneBytes3);
                tma_load_4d(smem + sl * kPlane3, &M.tm, x0 - 4, y0 - 4, z0 - 4 + k, vol_cur, &full[sl]);
                ++issued;
                if (++sl == kRing) {
                    sl = 0;
                    if (k + 1 >= 2 * kRing) eph ^= 1u;
                }
            }
            // the last load of every slot must have landed before the CTA may exit
            for (int q = max(0, issued - kRing); q < issued; ++q)
                (void)mbar_wait_bounded(&full[q % kRing], (uint32_t)((q / kRing) & 1));
        }
    } else if (!skip) {  // ---------------- consumer warps
        const int lx = (tid & 15) << 2, ly = tid >> 4;
        const int x = x0 + lx, y = y0 + ly;
        const bool col_ok = (x < M.Nx) && (y < M.Ny);
        float4 Gc, Ac;
        sponge_col3(M, y, x, Gc, Ac);
        const int sz = inc ? M.src[3 * shot] : -1;
        const int sy = inc ? M.src[3 * shot + 1] : -1;
        const int sx = inc ? M.src[3 * shot + 2] : -1;
        const float fsrc = inc ? M.wavelet[n] * M.vol_inv : 0.f;
        const long long plane_stride = (long long)M.Ny * M.P;
        const long long off0 = ((long long)z0 * M.Ny + y) * M.P + x;
        const int cell = ly * kTX + lx;
        const uint32_t dslot0 = smem_u32(dslots + cell);  // this thread's cells in Dtt slot 0
        int slot_c = 4, slot_w = 8;
        uint32_t ph_w = 0;
        int dj = 0;
        uint32_t dph = 0;  // Dtt slot and the parity of its current use
        for (int iz = 0; iz < nloc; ++iz) {
            const int z = z0 + iz;
            const long long off = off0 + (long long)iz * plane_stride;
            Pw3 cur_pw;
            if (col_ok) {
                cur_pw.s = ld4(M.s + off);
                cur_pw.prev = ld4(outv + off);
                if (!inc) cur_pw.dm = ld4(M.dm + (long long)b * F + off);
                if (iz + kPrefetch3 < nloc) {
                    const long long o2 = off + kPrefetch3 * plane_stride;
                    prefetch_l2(M.s + o2);
                    prefetch_l2(outv + o2);
                    if (!inc) prefetch_l2(M.dm + (long long)b * F + o2);
                }
            }
            bool ok = true;
            const int kfirst = (iz == 0) ? 0 : iz + 8;
            for (int k = kfirst; k <= iz + 8 && ok; ++k)
                ok = (iz == 0) ? mbar_wait_bounded(&full[k], 0u) : mbar_wait_bounded(&full[slot_w], ph_w);
            if (inc) {
                // the Born CTAs are done with the previous contents of Dtt slot dj
                if (ok && iz >= kDslots) ok = mbar_wait_bounded(&dempty[dj], dph ^ 1u);
                if (!ok) {
                    set_dev_error(p.err, DEVERR_TIMEOUT);
                    break;
                }
                float4 dw = make_float4(0.f, 0.f, 0.f, 0.f);
                if (col_ok)
                    cells3<STEP3_INC, false>(M, smem, slot_c, lx, ly, x, y, z, off, shot, 0, F, outv, cur_pw, Gc, Ac,
                                             sz, sy, sx, fsrc, false, make_float4(0.f, 0.f, 0.f, 0.f), &dw, nullptr);
                // every thread stores its 16 bytes (zeros off the grid) so that each Born CTA's
                // slot barrier receives exactly one plane, kTile3 * 4 bytes
                const uint32_t la = dslot0 + (uint32_t)(dj * kTile3 * 4);
                const uint32_t lb = smem_u32(&dfull[dj]);
                for (int r = 1; r <= nb; ++r) st_async4(mapa_rank(la, (uint32_t)r), dw, mapa_rank(lb, (uint32_t)r));
            } else {
                if (ok) {  // receivers of this plane, from its staged tile
                    const int rbeg = srec[iz], rend = srec[iz + 1];
                    if (rend > rbeg) {
                        const float* cur = smem + slot_c * kPlane3;
                        float* dout = M.data + (long long)shot * M.dss + (long long)b * M.dts + (long long)n * M.nr;
                        for (int i = rbeg + tid; i < rend; i += kThreads) {
                            const int r = M.rec_idx[i];
                            dout[r] = cur[(M.rec_zyx[3 * r + 1] - y0 + 4) * kHX3 + (M.rec_zyx[3 * r + 2] - x0 + 4)];
                        }
                    }
                }
                if (ok) ok = mbar_wait_bounded(&dfull[dj], dph);
                if (!ok) {
                    set_dev_error(p.err, DEVERR_TIMEOUT);
                    break;
                }
                // this slot's next plane: arm its barrier once the present one has completed
                if (tid == 0 && iz + kDslots < nloc) mbar_arm_tx(&dfull[dj], kTile3 * 4);
                if (col_ok) {
                    cur_pw.d = ld4(dslots + dj * kTile3 + cell);
                    cells3<STEP3_BORN, false>(M, smem, slot_c, lx, ly, x, y, z, off, shot, b, F, outv, cur_pw, Gc,
                                              Ac, -1, -1, -1, 0.f, false, make_float4(0.f, 0.f, 0.f, 0.f), nullptr,
                                              nullptr);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(mapa_rank(smem_u32(&dempty[dj]), 0u));
            }
            __syncwarp();
            if (lane == 0) {  // this warp is done with plane k = iz (the bottom of its window)
                int sf = slot_c - 4;
                sf += (sf < 0) ? kRing : 0;
                mbar_arrive(&empty[sf]);
            }
            slot_c = (slot_c + 1 == kRing) ? 0 : slot_c + 1;
            if (++slot_w == kRing) {
                slot_w = 0;
                ph_w ^= 1u;
            }
            if (++dj == kDslots) {
                dj = 0;
                dph ^= 1u;
            }
        }
    }
    __syncwarp();
    cluster_sync_all();  // no CTA of the cluster leaves while another may still reach its memory
}

cudaError_t launch_fwd3d_cluster(const StepParams3D& p, cudaStream_t st) {
    const ModelStep3D& M = p.m2;
    const int nf = M.nfield + 1;
    if (nf < 2 || nf > kMaxCluster3) return cudaErrorInvalidValue;
    dim3 grid(M.tiles_x * M.tiles_y * M.zchunks * nf, M.nshots);
    if (grid.y == 0) return cudaSuccess;
    const size_t sm = fwd3d_cluster_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_fwd3d_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kWs3Threads, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)nf;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fwd3d_cl, p);
}

// ---------------------------------------------------------------------------------------------
// Adjoint step with imaging on a cluster of G shots.
//
// A cluster holds the CTAs of one column tile and one trial for G consecutive shots of a wave
// (cluster rank = shot within the group).  Each CTA advances its shot's adjoint field exactly as
// k_step3d<ADJ> (same per-cell arithmetic, cells3) and forms its imaging term
// t_s = -Dtt u_s^{n-1} mu_s^n.  The image of the group is updated once per plane instead of once
// per shot: plane iz belongs to rank o = iz mod G, every other rank stores its t_s for that plane
// into rank o's reduction slot (distributed shared memory) with asynchronous stores that complete
// on o's slot barrier; rank o sums the G terms in rank order and applies one Kahan-compensated
// update to the group image [group][trial] in HBM, then releases the slot (plain arrivals).  Per cell, step and (shot, trial) the image
// read-modify-write (16 bytes with Kahan) thus costs 16/G bytes.  The receiver injection R^T r^n
// comes from the segment's prebuilt buffer of the planes that hold receivers (one float4 per
// thread on those planes), so no barrier of the whole CTA is taken.  Every wait is bounded.
// ---------------------------------------------------------------------------------------------
// Reduction planes per CTA: (G - 1) contributor planes for each of R slots (R = 1: a rank may run at
// most G planes ahead of the owner that last read its slot).  G = 1 and 2 keep the shared memory
// of a CTA within a third of the SM's, so three CTAs (27 warps) share an SM, as for the one-field
// kernels; G = 4 and 8 fit two.
template <int G>
struct AdjCl {
    static constexpr int R = 1;
    static constexpr int kRed = (G - 1) * R;
    static constexpr int kMinBlocks = (G <= 2) ? 3 : 2;
};

size_t adj3d_cluster_smem_bytes(int G) { return (size_t)kRing * kPlaneBytes3 + (size_t)(G - 1) * kTile3 * 4; }

template <int G, bool KAHAN>
__global__ void __launch_bounds__(kWs3Threads, AdjCl<G>::kMinBlocks) k_adj3d_cl(const __grid_constant__ StepParams3D p) {
    constexpr int R = AdjCl<G>::R;  // reduction slots per owner
    extern __shared__ __align__(128) float smem[];  // ring, then reduction planes [R][G - 1][kTile3]
    __shared__ __align__(8) uint64_t full[kRing], empty[kRing], rfull[R], wok[G][R];
    __shared__ int sband[kZCMax3D];  // receiver plane (band) index of each plane of the chunk, -1 without
    const ModelStep3D& M = p.m;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = (int)(blockIdx.x % M.nfield);
    int t = (int)(blockIdx.x / M.nfield);
    const int txi = t % M.tiles_x;
    t /= M.tiles_x;
    const int tyi = t % M.tiles_y;
    const int zc = t / M.tiles_y;
    const int x0 = txi * kTX, y0 = tyi * kTY3, z0 = zc * M.ZC;
    const int zend = min(z0 + M.ZC, M.Nz);
    const int shot = blockIdx.y;
    const int crank = (G > 1) ? (int)cluster_ctarank() : 0;  // == shot % G
    const int grp = shot / G;
    const int n = p.n;
    const int pc = (n + 1) & 1, po = pc ^ 1;
    const long long F = M.F;
    const int vol_cur = shot * M.nvol_shot + 2 * b + pc;
    float* outv = M.state + (long long)(shot * M.nvol_shot + 2 * b + po) * F;
    float* imgp = M.img + (long long)(grp * M.nfield + b) * F;
    float* cmpp = M.comp + (long long)(grp * M.nfield + b) * F;
    const int nloc = zend - z0;
    const int nplanes = nloc + 8;
    float* red = smem + kRing * kPlane3;

    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kThreads / 32);
        }
        for (int j = 0; j < R; ++j) {
            mbar_init(&rfull[j], 1);  // armed for the G - 1 other ranks' asynchronous stores of one plane
            if (G > 1) mbar_arm_tx(&rfull[j], (G - 1) * kTile3 * 4);
            for (int o = 0; o < G; ++o) mbar_init(&wok[o][j], kThreads / 32);  // rank o's consumer warps
        }
        fence_mbar_init();
    }
    if (tid < nloc) sband[tid] = M.rrow ? M.rrow[z0 + tid] : -1;
    __syncthreads();
    if (G > 1) cluster_sync_all();
    const bool skip = *reinterpret_cast<volatile int*>(p.err) != 0;

    if (warp == kThreads / 32) {  // ---------------- producer warp
        if (lane == 0 && !skip) {
            int sl = 0, issued = 0;
            uint32_t eph = 0;
            for (int k = 0; k < nplanes; ++k) {
                if (k >= kRing && !mbar_wait_bounded(&empty[sl], eph)) {
                    set_dev_error(p.err, DEVERR_TIMEOUT);
                    break;
                }
                mbar_expect_tx(&full[sl], kPlaneBytes3);
                tma_load_4d(smem + sl * kPlane3, &M.tm, x0 - 4, y0 - 4, z0 - 4 + k, vol_cur, &full[sl]);
                ++issued;
                if (++sl == kRing) {
                    sl = 0;
                    if (k + 1 >= 2 * kRing) eph ^= 1u;
                }
            }
            for (int q = max(0, issued - kRing); q < issued; ++q)
                (void)mbar_wait_bounded(&full[q % kRing], (uint32_t)((q / kRing) & 1));
        }
    } else if (!skip) {  // ---------------- consumer warps
        const int lx = (tid & 15) << 2, ly = tid >> 4;
        const int x = x0 + lx, y = y0 + ly;
        const bool col_ok = (x < M.Nx) && (y < M.Ny);
        float4 Gc, Ac;
        sponge_col3(M, y, x, Gc, Ac);
        const long long plane_stride = (long long)M.Ny * M.P;
        const long long off0 = ((long long)z0 * M.Ny + y) * M.P + x;
        const float* Din = M.Din + (long long)shot * M.Din_shot_stride;
        const int cell = ly * kTX + lx;
        const long long plane_cells = (long long)M.Ny * M.P;  // one band plane of the injection buffer
        const float* injp = M.inj + ((long long)(M.inj_slot * M.nshots + shot) * M.nfield + b) * M.inj_block +
                            (long long)y * M.P + x;
        int slot_c = 4, slot_w = 8;
        uint32_t ph_w = 0;
        for (int iz = 0; iz < nloc; ++iz) {
            const int z = z0 + iz;
            const long long off = off0 + (long long)iz * plane_stride;
            const int owner = iz % G;
            const bool own = (owner == crank);
            const int kk = iz / G;              // the owner's kk-th plane
            const int j = kk % R;               // its reduction slot
            const uint32_t use = (uint32_t)(kk / R);
            Pw3 cur_pw;
            if (col_ok) {
                cur_pw.s = ld4(M.s + off);
                cur_pw.prev = ld4(outv + off);
                cur_pw.d = ld4(Din + off);
                if (own) {
                    cur_pw.img = ld4(imgp + off);
                    if (KAHAN) cur_pw.cmp = ld4(cmpp + off);
                }
                if (iz + kPrefetch3 < nloc) {
                    const long long o2 = off + kPrefetch3 * plane_stride;
                    prefetch_l2(M.s + o2);
                    prefetch_l2(outv + o2);
                    prefetch_l2(Din + o2);
                    if ((iz + kPrefetch3) % G == crank) {
                        prefetch_l2(imgp + o2);
                        if (KAHAN) prefetch_l2(cmpp + o2);
                    }
                }
            }
            bool ok = true;
            const int kfirst = (iz == 0) ? 0 : iz + 8;
            for (int k = kfirst; k <= iz + 8 && ok; ++k)
                ok = (iz == 0) ? mbar_wait_bounded(&full[k], 0u) : mbar_wait_bounded(&full[slot_w], ph_w);
            if (!ok) {
                set_dev_error(p.err, DEVERR_TIMEOUT);
                break;
            }
            const int band = sband[iz];
            const bool inj = band >= 0;
            const float4 injv = (inj && col_ok) ? ld4(injp + band * plane_cells) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 tv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (col_ok)
                cells3<STEP3_ADJ, KAHAN>(M, smem, slot_c, lx, ly, x, y, z, off, shot, b, F, outv, cur_pw, Gc, Ac, -1,
                                         -1, -1, 0.f, inj, injv, nullptr, &tv);
            if (!own) {  // hand the term to the plane's owner (16 bytes per thread, zeros off the grid)
                if (use > 0 && !mbar_wait_bounded(&wok[owner][j], (use - 1u) & 1u)) {
                    set_dev_error(p.err, DEVERR_TIMEOUT);
                    break;
                }
                const int slot = j * (G - 1) + (crank < owner ? crank : crank - 1);  // contributor plane
                st_async4(mapa_rank(smem_u32(red + slot * kTile3 + cell), (uint32_t)owner), tv,
                          mapa_rank(smem_u32(&rfull[j]), (uint32_t)owner));
            } else {
                if (G > 1 && !mbar_wait_bounded(&rfull[j], use & 1u)) {
                    set_dev_error(p.err, DEVERR_TIMEOUT);
                    break;
                }
                // the slot's next use (G R planes on): arm once the present one has completed
                if (G > 1 && tid == 0 && iz + G * R < nloc) mbar_arm_tx(&rfull[j], (G - 1) * kTile3 * 4);
                if (col_ok) {
                    const float* rj = red + j * (G - 1) * kTile3 + cell;
                    float4 sum = (crank == 0) ? tv : ld4(rj);  // terms in rank order
#pragma unroll
                    for (int c = 1; c < G; ++c) {
                        const float4 v = (c == crank) ? tv : ld4(rj + (c < crank ? c : c - 1) * kTile3);
                        sum.x = __fadd_rn(sum.x, v.x);
                        sum.y = __fadd_rn(sum.y, v.y);
                        sum.z = __fadd_rn(sum.z, v.z);
                        sum.w = __fadd_rn(sum.w, v.w);
                    }
                    float4 iv = cur_pw.img;
                    if (KAHAN) {
                        float4 cv = cur_pw.cmp;
                        kahan4(iv, cv, sum.x, sum.y, sum.z, sum.w);
                        st4(cmpp + off, cv);
                    } else {
                        iv.x = __fadd_rn(iv.x, sum.x);
                        iv.y = __fadd_rn(iv.y, sum.y);
                        iv.z = __fadd_rn(iv.z, sum.z);
                        iv.w = __fadd_rn(iv.w, sum.w);
                    }
                    st4(imgp + off, iv);
                }
                if (G > 1) {
                    __syncwarp();
                    if (lane == 0)
                        for (int c = 0; c < G; ++c)
                            if (c != crank) mbar_arrive_remote(mapa_rank(smem_u32(&wok[crank][j]), (uint32_t)c));
                }
            }
            __syncwarp();
            if (lane == 0) {
                int sf = slot_c - 4;
                sf += (sf < 0) ? kRing : 0;
                mbar_arrive(&empty[sf]);
            }
            slot_c = (slot_c + 1 == kRing) ? 0 : slot_c + 1;
            if (++slot_w == kRing) {
                slot_w = 0;
                ph_w ^= 1u;
            }
        }
    }
    __syncwarp();
    if (G > 1) cluster_sync_all();
}

template <int G, bool KAHAN>
static cudaError_t launch_adj3d_cl_t(const StepParams3D& p, cudaStream_t st) {
    const ModelStep3D& M = p.m;
    dim3 grid(M.tiles_x * M.tiles_y * M.zchunks * M.nfield, M.nshots);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    if (grid.y % G) return cudaErrorInvalidValue;
    const size_t sm = adj3d_cluster_smem_bytes(G);
    cudaError_t e = cudaFuncSetAttribute(k_adj3d_cl<G, KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kWs3Threads, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = (unsigned)G;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_adj3d_cl<G, KAHAN>, p);
}

cudaError_t launch_adj3d_cluster(int G, bool kahan, const StepParams3D& p, cudaStream_t st) {
    switch (G) {
        case 1: return kahan ? launch_adj3d_cl_t<1, true>(p, st) : launch_adj3d_cl_t<1, false>(p, st);
        case 2: return kahan ? launch_adj3d_cl_t<2, true>(p, st) : launch_adj3d_cl_t<2, false>(p, st);
        case 4: return kahan ? launch_adj3d_cl_t<4, true>(p, st) : launch_adj3d_cl_t<4, false>(p, st);
        case 8: return kahan ? launch_adj3d_cl_t<8, true>(p, st) : launch_adj3d_cl_t<8, false>(p, st);
    }
    return cudaErrorInvalidValue;
}

template <int MODE, bool PROD>
static cudaError_t launch3_ws(const StepParams3D& p, dim3 grid, cudaStream_t st) {
    const size_t sm = (size_t)kRing * kPlaneBytes3;
    // set on every launch (a host-side attribute, no stream work): no shared state between threads
    cudaError_t e =
        cudaFuncSetAttribute(k_step3d_ws<MODE, PROD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_step3d_ws<MODE, PROD><<<grid, PROD ? kWs3Threads : kThreads, sm, st>>>(p);
    return cudaGetLastError();
}

template <int MODE, bool KAHAN>
static cudaError_t launch3(const StepParams3D& p, dim3 grid, cudaStream_t st) {
    const size_t sm = step3d_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_step3d<MODE, KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_step3d<MODE, KAHAN><<<grid, kThreads, sm, st>>>(p);
    return cudaGetLastError();
}

template <bool PROD>
static cudaError_t launch3_ws_mode(int mode, bool kahan, const StepParams3D& p, dim3 grid, cudaStream_t st,
                                   bool* done) {
    *done = true;
    switch (mode) {
        case STEP3_INC: return launch3_ws<STEP3_INC, PROD>(p, grid, st);
        case STEP3_INC_SAMPLE: return launch3_ws<STEP3_INC_SAMPLE, PROD>(p, grid, st);
        case STEP3_BORN: return launch3_ws<STEP3_BORN, PROD>(p, grid, st);
        case STEP3_ADJ:  // the per-step Kahan adjoint keeps the one-barrier-per-plane kernel
            if (!kahan) return launch3_ws<STEP3_ADJ, PROD>(p, grid, st);
            break;
        default: break;
    }
    *done = false;
    return cudaSuccess;
}

cudaError_t launch_step3d(int mode, bool kahan, int pipeline, const StepParams3D& p, cudaStream_t st) {
    const ModelStep3D& M = p.m;
    dim3 grid(M.tiles_x * M.tiles_y * M.zchunks * M.nfield, M.nshots);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    if (pipeline) {  // 2: producer warp; 3: the last compute warp out of a slot refills it
        bool done = false;
        const cudaError_t e = (pipeline == 3) ? launch3_ws_mode<false>(mode, kahan, p, grid, st, &done)
                                              : launch3_ws_mode<true>(mode, kahan, p, grid, st, &done);
        if (done) return e;
    }
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
