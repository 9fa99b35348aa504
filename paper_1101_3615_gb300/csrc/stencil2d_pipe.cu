// Warp-specialised, TMA-pipelined 2D time-step kernels (sm_103a).
//
// The plain kernels of stencil2d.cu give every CTA one tile (load, wait,
// compute, store), so each CTA exposes the full load latency.  Here a
// persistent CTA walks a list of work groups -- one field of one 64 x 16 tile:
// the incident field, one Born field, or one adjoint field of one shot -- with
//   * one producer warp that decodes the next group, writes its descriptor to
//     shared memory and issues its TMA loads into an S-stage ring: the radius-4
//     halo tile of the differentiated field (72 x 24) and up to three plain
//     64 x 16 tiles of pointwise operands (previous level, s, dm, Dtt); for
//     adjoint tiles that hold receivers it also assembles the injection tile;
//   * eight consumer warps that wait on the stage's "full" mbarrier, compute,
//     store from registers, and release the stage through its "empty"
//     mbarrier (one arrival per warp).
// There is no CTA-wide barrier in the main loop; a sentinel descriptor ends
// the list.  Every wait is bounded (2 s of %globaltimer) and reports through
// the device error word.  Arithmetic, boundary handling and the adjoint form
// are those of stencil2d.cu.
#include "common.cuh"
#include "internal.h"

namespace probe {

namespace {

constexpr int TZ = kPipeTZ;
constexpr int HX = kTX + 8;
constexpr int HZ = TZ + 8;
constexpr int HALO = HX * HZ;   // floats
constexpr int PLAIN = kTX * TZ; // floats
constexpr int FWD_STAGE = HALO + 2 * PLAIN;
constexpr int ADJ_STAGE = HALO + 4 * PLAIN;  // + injection tile
constexpr unsigned HALO_B = HALO * 4u, PLAIN_B = PLAIN * 4u;
constexpr int kConsumerWarps = kThreads / 32;     // 8
constexpr int kWsThreads = kThreads + 32;        // + producer warp

struct Group {
    int mi, unit, tile, x0, z0;
    int f;      // forward: field (0 incident, 1.. Born trial + 1); adjoint: shot-in-group * NBC + trial-in-chunk
    int last;   // adjoint: last group of its item
    int inj;    // adjoint: injection tile present
    int sz, sx; // forward: source cell of the shot
    int rbeg, rend;  // receivers of the tile (CSR range)
    float fsrc; // forward: w[n] / (hz hx)
};

__device__ __forceinline__ int model_of(const StepParams2D& p, int item) {
    int mi = 0;
#pragma unroll
    for (int k = 1; k < kMaxModels; ++k)
        if (k < p.nmodels && item >= p.m[k].item_begin) mi = k;
    return mi;
}

__device__ __forceinline__ void sponge_fac(const ModelStep2D& M, int z, int x, float& G, float& am) {
    const int rz = max(max(M.pad - z, z - (M.pad + M.nz - 1)), 0);
    const int rx = max(max(M.pad - x, x - (M.pad + M.nx - 1)), 0);
    sponge_pair(__fmaf_rn(M.cz, (float)(rz * rz), __fmul_rn(M.cx, (float)(rx * rx))), G, am);
}

// Laplacian of 4 cells at halo-tile coordinates (row, col); first-difference x taps.
__device__ __forceinline__ void lap4p(const float* t, int row, int col, const ModelStep2D& M, float4& center,
                                      float L[4]) {
    const float* rp = t + row * HX + col;
    const float4 a = ld4(rp - 4), b = ld4(rp), c = ld4(rp + 4);
    const float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    center = b;
    float d[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) d[i] = v[i + 1] - v[i];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float acc = M.cxm[0] * (d[4 + j] - d[3 + j]);
#pragma unroll
        for (int m = 1; m < 4; ++m) acc = fmaf(M.cxm[m], d[4 + j + m] - d[3 + j - m], acc);
        L[j] = acc;
    }
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        const float4 up = ld4(rp - k * HX), dn = ld4(rp + k * HX);
        const float w = M.lz[k - 1];
        L[0] = fmaf(w, (up.x - b.x) + (dn.x - b.x), L[0]);
        L[1] = fmaf(w, (up.y - b.y) + (dn.y - b.y), L[1]);
        L[2] = fmaf(w, (up.z - b.z) + (dn.z - b.z), L[2]);
        L[3] = fmaf(w, (up.w - b.w) + (dn.w - b.w), L[3]);
    }
}

__device__ __forceinline__ Group decode(const StepParams2D& p, int item) {
    Group q;
    q.mi = model_of(p, item);
    const ModelStep2D& M = p.m[q.mi];
    const int r = item - M.item_begin;
    q.unit = r / M.ntiles;
    q.tile = r - q.unit * M.ntiles;
    const int tz = q.tile / M.tiles_x;
    q.z0 = tz * TZ;
    q.x0 = (q.tile - tz * M.tiles_x) * kTX;
    q.f = 0;
    q.last = 0;
    q.inj = 0;
    return q;
}

__device__ __forceinline__ void fail_exit(int* err) { set_dev_error(err, DEVERR_TIMEOUT); }

// ---- forward ---------------------------------------------------------------
template <int KIND, int S, bool MULTI>
__global__ void __launch_bounds__(kWsThreads) k_fwd2d_ws(const __grid_constant__ StepParams2D p) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ Group info[S];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int total = p.total_items;
    const int n = p.n;
    const int pc = n & 1, po = pc ^ 1;
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kConsumerWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kConsumerWarps) {  // ---------------- producer warp
        if (lane != 0) return;
        int g = 0;
        for (int item = blockIdx.x;; item += gridDim.x) {
            const bool done = item >= total;
            Group q = done ? Group{} : decode(p, item);
            const int ngr = done ? 1 : (KIND == FWD_BORN ? 1 + p.m[q.mi].nb : 1);
            for (int f = 0; f < ngr; ++f, ++g) {
                const int s = g % S;
                if (g >= S && !mbar_wait_bounded(&empty[s], (uint32_t)(((g / S) - 1) & 1))) {
                    fail_exit(p.err);
                    return;
                }
                if (done) {
                    info[s].f = -1;  // sentinel
                    mbar_arrive(&full[s]);
                    return;
                }
                const ModelStep2D& M = p.m[q.mi];
                q.f = f;
                if (f == 0) {
                    q.sz = M.src_zx[2 * q.unit];
                    q.sx = M.src_zx[2 * q.unit + 1];
                    q.fsrc = M.wavelet[n] * M.vol_inv;
                    q.rbeg = M.rec_tile_ptr[q.tile];
                    q.rend = M.rec_tile_ptr[q.tile + 1];
                }  // later fields of the same item keep these values
                info[s] = q;
                float* st = smem + s * FWD_STAGE;
                mbar_expect_tx(&full[s], HALO_B + 2 * PLAIN_B);
                if (f == 0) {
                    tma_load_3d(st, &M.tm_u, q.x0 - 4, q.z0 - 4, q.unit * 2 + pc, &full[s]);
                    tma_load_3d(st + HALO, &M.tm_sp, q.x0, q.z0, 0, &full[s]);
                    tma_load_3d(st + HALO + PLAIN, &M.tm_up, q.x0, q.z0, q.unit * 2 + po, &full[s]);
                } else {
                    const int b = f - 1;
                    const int pl = (q.unit * M.nb + b) * 2;
                    tma_load_3d(st, &M.tm_f, q.x0 - 4, q.z0 - 4, pl + pc, &full[s]);
                    tma_load_3d(st + HALO, &M.tm_dmp, q.x0, q.z0, b, &full[s]);
                    tma_load_3d(st + HALO + PLAIN, &M.tm_fp, q.x0, q.z0, pl + po, &full[s]);
                }
            }
        }
    }

    // ---------------- consumer warps
    const int lx = (tid & 15) << 2, lz = tid >> 4;
    float4 sv = make_float4(0.f, 0.f, 0.f, 0.f);
    float D[4] = {0.f, 0.f, 0.f, 0.f};
    bool interior = false;
    for (int g = 0;; ++g) {
        const int s = g % S;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((g / S) & 1))) {
            fail_exit(p.err);
            return;
        }
        const Group q = info[s];
        if (q.f < 0) return;
        const ModelStep2D& M = p.m[MULTI ? q.mi : 0];  // single model: loop-invariant descriptor
        const float* st = smem + s * FWD_STAGE;
        const int shot = q.unit;
        const int x = q.x0 + lx, z = q.z0 + lz;
        const bool valid = (z < M.Nz) && (x < M.Nx);
        const bool full_w = (q.x0 + kTX <= M.Nx);
        const long long off = (long long)z * M.P + x;
        float L[4];
        float4 c;
        lap4p(st, lz + 4, lx + 4, M, c, L);
        const float4 pa = ld4(st + HALO + lz * kTX + lx);
        const float4 pold = ld4(st + HALO + PLAIN + lz * kTX + lx);
        float o[4];
        if (q.f == 0) {
            interior = (z >= M.pad) && (z < M.pad + M.nz) && (x >= M.pad) && (x + 3 < M.pad + M.nx);
            sv = pa;
            if (z == q.sz) {
                const int j = q.sx - x;
                if (j >= 0 && j < 4) L[j] += q.fsrc;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float Fo = __fmul_rn(get(sv, j), L[j]);
                D[j] = __fmul_rn(Fo, M.inv_dt2);
                float G = 1.f, am = 1.f;
                if (!interior) sponge_fac(M, z, x + j, G, am);
                o[j] = (full_w || x + j < M.Nx) ? leapfrog(G, get(c, j), am, get(pold, j), Fo) : 0.f;
            }
            if (valid) {
                st4(M.u + (long long)(shot * 2 + po) * M.F + off, make_float4(o[0], o[1], o[2], o[3]));
                if (KIND == FWD_INCIDENT_DTT || (KIND == FWD_BORN && M.dtt_store))
                    st4(M.dtt + (long long)shot * M.dtt_shot_stride + (long long)M.dtt_slot * M.F + off,
                        make_float4(D[0], D[1], D[2], D[3]));
            }
            if (KIND == FWD_INCIDENT_SAMPLE && q.rend > q.rbeg) {
                const int beg = q.rbeg, end = q.rend;
                float* out = M.data + (long long)shot * M.data_shot_stride + (long long)n * M.nr;
                for (int i = beg + tid; i < end; i += kThreads) {
                    const int r = M.rec_tile_idx[i];
                    out[r] = st[(M.rec_zx[2 * r] - q.z0 + 4) * HX + (M.rec_zx[2 * r + 1] - q.x0 + 4)];
                }
            }
        } else {
            const int b = q.f - 1;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float G = 1.f, am = 1.f;
                if (!interior) sponge_fac(M, z, x + j, G, am);
                const float src = __fmaf_rn(-get(pa, j), D[j], L[j]);
                o[j] = (full_w || x + j < M.Nx) ? leapfrog(G, get(c, j), am, get(pold, j), __fmul_rn(get(sv, j), src))
                                                : 0.f;
            }
            if (valid)
                st4(M.f + (long long)((shot * M.nb + b) * 2 + po) * M.F + off, make_float4(o[0], o[1], o[2], o[3]));
            const int beg = q.rbeg, end = q.rend;
            if (end > beg) {
                float* out = M.data + (long long)shot * M.data_shot_stride + (long long)b * M.data_trial_stride +
                             (long long)n * M.nr;
                for (int i = beg + tid; i < end; i += kThreads) {
                    const int r = M.rec_tile_idx[i];
                    out[r] = st[(M.rec_zx[2 * r] - q.z0 + 4) * HX + (M.rec_zx[2 * r + 1] - q.x0 + 4)];
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ---- adjoint ---------------------------------------------------------------
// Item = (model, shot group, tile); its groups are (shot jj of the group, trial bi of the chunk).
template <int NBC, bool KAHAN, int S, bool MULTI>
__global__ void __launch_bounds__(kWsThreads) k_adj2d_ws(const __grid_constant__ StepParams2D p) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ Group info[S];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int total = p.total_items;
    const int n = p.n;
    const int pc = (n + 1) & 1, po = n & 1;
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kConsumerWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kConsumerWarps) {  // ---------------- producer warp
        int g = 0;
        for (int item = blockIdx.x;; item += gridDim.x) {
            const bool done = item >= total;
            Group q = done ? Group{} : decode(p, item);
            int nsh = 1, nbc = 1;
            if (!done) {
                const ModelStep2D& M = p.m[q.mi];
                nsh = min(M.shot_group, M.nshots - q.unit * M.shot_group);
                nbc = min(NBC, M.nb - M.chunk * NBC);
            }
            for (int jj = 0; jj < nsh; ++jj) {
                for (int bi = 0; bi < nbc; ++bi, ++g) {
                    const int s = g % S;
                    bool ok = true;
                    if (lane == 0 && g >= S) ok = mbar_wait_bounded(&empty[s], (uint32_t)(((g / S) - 1) & 1));
                    if (!__shfl_sync(0xffffffffu, ok, 0)) {
                        if (lane == 0) fail_exit(p.err);
                        return;
                    }
                    if (done) {
                        if (lane == 0) {
                            info[s].f = -1;
                            mbar_arrive(&full[s]);
                        }
                        return;
                    }
                    const ModelStep2D& M = p.m[q.mi];
                    float* st = smem + s * ADJ_STAGE;
                    const int shot = q.unit * M.shot_group + jj;
                    const int b = M.chunk * NBC + bi;
                    const int rbeg = M.rec_tile_ptr[q.tile], rend = M.rec_tile_ptr[q.tile + 1];
                    const bool inj = rend > rbeg;
                    if (inj) {  // R^T r^n of this tile, assembled by the producer warp
                        float* it = st + HALO + 3 * PLAIN;
                        for (int i = lane; i < PLAIN; i += 32) it[i] = 0.f;
                        __syncwarp();
                        const float* rr = M.rdata + (long long)shot * M.data_shot_stride +
                                          (long long)b * M.data_trial_stride + (long long)n * M.nr;
                        for (int i = rbeg + lane; i < rend; i += 32) {
                            const int rcv = M.rec_tile_idx[i];
                            atomicAdd(&it[(M.rec_zx[2 * rcv] - q.z0) * kTX + (M.rec_zx[2 * rcv + 1] - q.x0)], rr[rcv]);
                        }
                        __syncwarp();
                    }
                    if (lane == 0) {
                        Group gi = q;
                        gi.f = jj * NBC + bi;
                        gi.last = (jj == nsh - 1) && (bi == nbc - 1);
                        gi.inj = inj;
                        info[s] = gi;
                        const int pl = (shot * M.nb + b) * 2;
                        mbar_expect_tx(&full[s], HALO_B + 3 * PLAIN_B);
                        tma_load_3d(st, &M.tm_f, q.x0 - 4, q.z0 - 4, pl + pc, &full[s]);
                        tma_load_3d(st + HALO, &M.tm_fp, q.x0, q.z0, pl + po, &full[s]);
                        tma_load_3d(st + HALO + PLAIN, &M.tm_dtp, q.x0, q.z0, shot * M.dtt_slots + M.dtt_slot,
                                    &full[s]);
                        tma_load_3d(st + HALO + 2 * PLAIN, &M.tm_sp, q.x0, q.z0, 0, &full[s]);
                    }
                    __syncwarp();
                }
            }
        }
    }

    // ---------------- consumer warps
    const int lx = (tid & 15) << 2, lz = tid >> 4;
    float acc[NBC][4];
#pragma unroll
    for (int k = 0; k < NBC; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[k][j] = 0.f;
    for (int g = 0;; ++g) {
        const int s = g % S;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((g / S) & 1))) {
            fail_exit(p.err);
            return;
        }
        const Group q = info[s];
        if (q.f < 0) return;
        const ModelStep2D& M = p.m[MULTI ? q.mi : 0];  // single model: loop-invariant descriptor
        const float* st = smem + s * ADJ_STAGE;
        const int jj = q.f / NBC, bi = q.f - (q.f / NBC) * NBC;
        const int shot = q.unit * M.shot_group + jj;
        const int b = M.chunk * NBC + bi;
        const int x = q.x0 + lx, z = q.z0 + lz;
        const bool valid = (z < M.Nz) && (x < M.Nx);
        const bool full_w = (q.x0 + kTX <= M.Nx);
        const bool interior = (z >= M.pad) && (z < M.pad + M.nz) && (x >= M.pad) && (x + 3 < M.pad + M.nx);
        const long long off = (long long)z * M.P + x;
        float L[4];
        float4 c;
        lap4p(st, lz + 4, lx + 4, M, c, L);
        const float4 mo = ld4(st + HALO + lz * kTX + lx);
        const float4 Dv = ld4(st + HALO + PLAIN + lz * kTX + lx);
        const float4 sv = ld4(st + HALO + 2 * PLAIN + lz * kTX + lx);
        if (q.inj) {
            const float4 iv = ld4(st + HALO + 3 * PLAIN + lz * kTX + lx);
            L[0] += iv.x;
            L[1] += iv.y;
            L[2] += iv.z;
            L[3] += iv.w;
        }
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float G = 1.f, am = 1.f;
            if (!interior) sponge_fac(M, z, x + j, G, am);
            o[j] = (full_w || x + j < M.Nx) ? leapfrog(G, get(c, j), am, get(mo, j), __fmul_rn(get(sv, j), L[j]))
                                            : 0.f;
        }
#pragma unroll
        for (int k = 0; k < NBC; ++k)
            if (k == bi) {
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[k][j] = fmaf(-get(Dv, j), o[j], acc[k][j]);
            }
        if (valid) st4(M.f + (long long)((shot * M.nb + b) * 2 + po) * M.F + off, make_float4(o[0], o[1], o[2], o[3]));
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (q.last) {  // image update of this item's shot group
            const int nbc = min(NBC, M.nb - M.chunk * NBC);
            if (valid) {
                float* img = M.img + (long long)q.unit * M.img_group_stride;
                float* cmp = M.comp + (long long)q.unit * M.img_group_stride;
#pragma unroll
                for (int k = 0; k < NBC; ++k) {
                    if (k < nbc) {
                        const long long boff = (long long)(M.chunk * NBC + k) * M.F + off;
                        float4 iv = ld4(img + boff);
                        float* ia = reinterpret_cast<float*>(&iv);
                        if (KAHAN) {
                            float4 cv = ld4(cmp + boff);
                            float* ca = reinterpret_cast<float*>(&cv);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float y = acc[k][j] - ca[j];
                                const float t = ia[j] + y;
                                ca[j] = (t - ia[j]) - y;
                                ia[j] = t;
                            }
                            st4(cmp + boff, cv);
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j) ia[j] += acc[k][j];
                        }
                        st4(img + boff, iv);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < NBC; ++k)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[k][j] = 0.f;
        }
    }
}

int occupancy(const void* fn, size_t smem) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kWsThreads, smem);
    return nb < 1 ? 1 : nb;
}

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

template <typename K>
cudaError_t launch_persistent(K kernel, size_t smem, int total, const StepParams2D& p, cudaStream_t st) {
    static_assert(sizeof(StepParams2D) < 32000, "kernel parameter block too large");
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(total, num_sms() * occupancy((const void*)kernel, smem));
    if (grid <= 0) return cudaSuccess;
    kernel<<<grid, kWsThreads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

size_t pipe_smem_bytes(int stages, bool adjoint) {
    return (size_t)stages * (adjoint ? ADJ_STAGE : FWD_STAGE) * 4;
}

cudaError_t launch_fwd2d_pipe(FwdKind kind, int stages, const StepParams2D& p, cudaStream_t st) {
    const int total = p.total_items;
    if (total <= 0) return cudaSuccess;
    const size_t sm = pipe_smem_bytes(stages, false);
#define PROBE_FWD_CASE(K)                                                                            \
    case K:                                                                                          \
        if (p.nmodels > 1)                                                                           \
            return stages == 4   ? launch_persistent(k_fwd2d_ws<K, 4, true>, sm, total, p, st)       \
                   : stages == 3 ? launch_persistent(k_fwd2d_ws<K, 3, true>, sm, total, p, st)       \
                                 : launch_persistent(k_fwd2d_ws<K, 2, true>, sm, total, p, st);      \
        return stages == 4   ? launch_persistent(k_fwd2d_ws<K, 4, false>, sm, total, p, st)          \
               : stages == 3 ? launch_persistent(k_fwd2d_ws<K, 3, false>, sm, total, p, st)          \
                             : launch_persistent(k_fwd2d_ws<K, 2, false>, sm, total, p, st);
    switch (kind) {
        PROBE_FWD_CASE(FWD_INCIDENT)
        PROBE_FWD_CASE(FWD_INCIDENT_DTT)
        PROBE_FWD_CASE(FWD_BORN)
        PROBE_FWD_CASE(FWD_INCIDENT_SAMPLE)
    }
#undef PROBE_FWD_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_adj2d_pipe(int nbc, bool kahan, int stages, const StepParams2D& p, int chunks, cudaStream_t st) {
    const int total = p.total_items;
    if (total <= 0) return cudaSuccess;
    const size_t sm = pipe_smem_bytes(stages, true);
    StepParams2D q = p;
    for (int c = 0; c < chunks; ++c) {
        for (int k = 0; k < q.nmodels; ++k) q.m[k].chunk = c;
        cudaError_t e;
#define PROBE_ADJ_SM(NB, KH, MU)                                                            \
    e = stages == 4   ? launch_persistent(k_adj2d_ws<NB, KH, 4, MU>, sm, total, q, st)      \
        : stages == 3 ? launch_persistent(k_adj2d_ws<NB, KH, 3, MU>, sm, total, q, st)      \
                      : launch_persistent(k_adj2d_ws<NB, KH, 2, MU>, sm, total, q, st);
#define PROBE_ADJ_S(NB, KH)            \
    if (q.nmodels > 1) {               \
        PROBE_ADJ_SM(NB, KH, true)     \
    } else {                           \
        PROBE_ADJ_SM(NB, KH, false)    \
    }
#define PROBE_ADJ(NB)           \
    if (kahan) {                \
        PROBE_ADJ_S(NB, true)   \
    } else {                    \
        PROBE_ADJ_S(NB, false)  \
    }
        switch (nbc) {
            case 1: PROBE_ADJ(1) break;
            case 2: PROBE_ADJ(2) break;
            case 4: PROBE_ADJ(4) break;
            case 8: PROBE_ADJ(8) break;
            default: return cudaErrorInvalidValue;
        }
#undef PROBE_ADJ
#undef PROBE_ADJ_S
#undef PROBE_ADJ_SM
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace probe
