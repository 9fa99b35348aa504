// Warp-specialised, TMA-pipelined 2D time-step kernels (sm_103a).
//
// The plain kernels of stencil2d.cu give every CTA one tile (load, wait,
// compute, store), so each CTA exposes the full load latency.  Here a
// persistent CTA walks a list of work groups -- one field of one 64 x 16R
// tile: the incident field, one Born field, or one adjoint field of one shot --
// with
//   * one producer warp that decodes the next group, writes its descriptor to
//     shared memory and issues its TMA loads into an S-stage ring: the radius-4
//     halo tile of the differentiated field ((64+8) x (16R+8)) and plain
//     64 x 16R tiles of the pointwise operands (previous level, s, dm, Dtt);
//     for adjoint tiles that hold receivers it also assembles the injection tile;
//   * eight consumer warps that wait on the stage's "full" mbarrier, compute,
//     store from registers, and release the stage through its "empty"
//     mbarrier (one arrival per warp).
// Each consumer thread owns R consecutive rows of 4 cells, so the z taps share
// their first differences across the rows (the same first-difference form as
// the x taps) and the per-group bookkeeping is spread over 4R cells.  Operands
// shared by the groups of one work item stay in registers: s and Dtt u^n of the
// incident step for the Born fields; s for all adjoint groups of an item and
// Dtt for all trials of one shot.  Tiles whose cells are all interior take a
// path without sponge or edge logic.
// There is no CTA-wide barrier in the main loop; a sentinel descriptor ends
// the list.  Every wait is bounded (2 s of %globaltimer) and reports through
// the device error word.  The arithmetic is that of stencil2d.cu operation for
// operation, so both kernel families give the same bits.
#include "common.cuh"
#include "internal.h"

namespace probe {

namespace {

constexpr int HX = kTX + 8;
constexpr int kConsumerWarps = kThreads / 32;  // 8
constexpr int kWsThreads = kThreads + 32;      // + producer warp

template <int R>
struct Ws {
    static constexpr int TZ = 16 * R;
    static constexpr int HZ = TZ + 8;
    static constexpr int HALO = HX * HZ;    // floats
    static constexpr int PLAIN = kTX * TZ;  // floats
    static constexpr int FWD_STAGE = HALO + 2 * PLAIN;
    // adjoint stage: halo of mu^{n+1}, mu^{n+2}, Dtt, s, and the image and compensation tiles of
    // a trial's last group
    static constexpr int ADJ_STAGE = HALO + 5 * PLAIN;
    static constexpr unsigned HALO_B = HALO * 4u, PLAIN_B = PLAIN * 4u;
};

struct Group {
    int mi, unit, tile, x0, z0;
    int f;      // forward: field (0 incident, 1.. Born trial + 1); adjoint: shot-in-group * NBC + trial-in-chunk;
                // -1 ends the list
    int last;   // adjoint: the group's last shot (the trial's image update happens here)
    int inj;    // adjoint: injection tile present
    int fast;   // every cell of the tile is an interior cell (no sponge, no grid edge)
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

// One cell of the time update; rhs = s (L + source) of the field.  Interior
// ("fast") tiles have G = a- = 1; elsewhere the sponge factors follow from the
// cell's distance to the interior, and columns past Nx are written as zero.
__device__ __forceinline__ float cell_update(const ModelStep2D& M, bool fast, int z, int x, float c, float prev,
                                             float rhs) {
    float G = 1.f, am = 1.f;
    if (!fast) {
        if (x >= M.Nx) return 0.f;
        const int rz = max(max(M.pad - z, z - (M.pad + M.nz - 1)), 0);
        const int rx = max(max(M.pad - x, x - (M.pad + M.nx - 1)), 0);
        sponge_pair(__fmaf_rn(M.cz, (float)(rz * rz), __fmul_rn(M.cx, (float)(rx * rx))), G, am);
    }
    return leapfrog(G, c, am, prev, rhs);
}

// Laplacian of R rows x 4 cells whose first cell sits at halo coordinates (row, col).
// Both axes in first-difference form: with d_i = v_{i+1} - v_i,
//   sum_k w_k (v_{c+k} + v_{c-k} - 2 v_c) = sum_{m=0..3} C_m (d_{c+m} - d_{c-m-1}),
//   C_m = sum_{k>m} w_k / h^2,
// x first (11 shared differences per row), then z (R + 7 shared differences per column).
// PACKED: z taps in packed FP32x2 (the forward kernels) or scalar (the adjoint, where the packed
// form measured slower); the two give the same bits.
template <int R, bool PACKED>
__device__ __forceinline__ void lap_rows(const float* t, int row, int col, const ModelStep2D& M, float4 c[R],
                                         float L[R][4]) {
    const float* rp = t + row * HX + col;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float4 a = ld4(rp + r * HX - 4), b = ld4(rp + r * HX), e = ld4(rp + r * HX + 4);
        c[r] = b;
        const float w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, e.x, e.y, e.z, e.w};
        float d[11];
#pragma unroll
        for (int i = 0; i < 11; ++i) d[i] = w[i + 1] - w[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float acc = M.cxm[0] * (d[4 + j] - d[3 + j]);
#pragma unroll
            for (int m = 1; m < 4; ++m) acc = fmaf(M.cxm[m], d[4 + j + m] - d[3 + j - m], acc);
            L[r][j] = acc;
        }
    }
    // z, outward: rows below the first cell row (lo) and above the last (hi) are loaded
    // as the tap index m grows; row r's term m is C_m ((v_{r+m+1} - v_{r+m}) - (v_{r-m} - v_{r-m-1})).
    // Differences between rows inside the block are formed once and shared by the R rows.
    if (!PACKED) {
        if (R == 1) {
            float4 lo = c[0], hi = c[0];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float4 dn = ld4(rp - (m + 1) * HX), up = ld4(rp + (m + 1) * HX);
                L[0][0] = fmaf(M.czm[m], (up.x - hi.x) - (lo.x - dn.x), L[0][0]);
                L[0][1] = fmaf(M.czm[m], (up.y - hi.y) - (lo.y - dn.y), L[0][1]);
                L[0][2] = fmaf(M.czm[m], (up.z - hi.z) - (lo.z - dn.z), L[0][2]);
                L[0][3] = fmaf(M.czm[m], (up.w - hi.w) - (lo.w - dn.w), L[0][3]);
                lo = dn;
                hi = up;
            }
        } else {
            const float4 c0 = c[0], c1 = c[R - 1];
            const float4 gin = make_float4(c1.x - c0.x, c1.y - c0.y, c1.z - c0.z, c1.w - c0.w);
            float4 lo = c0, hi = c1, glo = gin, ghi = gin;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float4 dn = ld4(rp - (m + 1) * HX), up = ld4(rp + (m + 2) * HX);
                const float4 gd = make_float4(lo.x - dn.x, lo.y - dn.y, lo.z - dn.z, lo.w - dn.w);
                const float4 gu = make_float4(up.x - hi.x, up.y - hi.y, up.z - hi.z, up.w - hi.w);
                L[0][0] = fmaf(M.czm[m], ghi.x - gd.x, L[0][0]);
                L[0][1] = fmaf(M.czm[m], ghi.y - gd.y, L[0][1]);
                L[0][2] = fmaf(M.czm[m], ghi.z - gd.z, L[0][2]);
                L[0][3] = fmaf(M.czm[m], ghi.w - gd.w, L[0][3]);
                L[R - 1][0] = fmaf(M.czm[m], gu.x - glo.x, L[R - 1][0]);
                L[R - 1][1] = fmaf(M.czm[m], gu.y - glo.y, L[R - 1][1]);
                L[R - 1][2] = fmaf(M.czm[m], gu.z - glo.z, L[R - 1][2]);
                L[R - 1][3] = fmaf(M.czm[m], gu.w - glo.w, L[R - 1][3]);
                lo = dn;
                hi = up;
                glo = gd;
                ghi = gu;
            }
        }
        return;
    }
    // (packed: the same subtractions and fused multiply-adds, two lanes per instruction)
    if (R == 1) {
        P4 acc = p4(L[0][0], L[0][1], L[0][2], L[0][3]);
        P4 lo = p4(c[0]), hi = lo;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const P4 dn = p4(ld4(rp - (m + 1) * HX)), up = p4(ld4(rp + (m + 1) * HX));
            const P4 w = p4(M.czm[m], M.czm[m], M.czm[m], M.czm[m]);
            acc = p4fma(w, p4sub(p4sub(up, hi), p4sub(lo, dn)), acc);
            lo = dn;
            hi = up;
        }
        const float4 o = f4(acc);
        L[0][0] = o.x;
        L[0][1] = o.y;
        L[0][2] = o.z;
        L[0][3] = o.w;
    } else {
        // R = 2: values v_{-4..5} relative to row 0; g_i = v_{i+1} - v_i.
        // row 0 term m: g_m - g_{-m-1}; row 1 term m: g_{m+1} - g_{-m}.
        P4 a0 = p4(L[0][0], L[0][1], L[0][2], L[0][3]), a1 = p4(L[R - 1][0], L[R - 1][1], L[R - 1][2], L[R - 1][3]);
        const P4 c0 = p4(c[0]), c1 = p4(c[R - 1]);
        const P4 gin = p4sub(c1, c0);  // g_0
        P4 lo = c0, hi = c1;           // current outermost rows below / above
        P4 glo = gin, ghi = gin;       // g_{-m} (row 1's lower) and g_m (row 0's upper) of the last step
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const P4 dn = p4(ld4(rp - (m + 1) * HX)), up = p4(ld4(rp + (m + 2) * HX));
            const P4 gd = p4sub(lo, dn);  // g_{-m-1}
            const P4 gu = p4sub(up, hi);  // g_{m+1}
            const P4 w = p4(M.czm[m], M.czm[m], M.czm[m], M.czm[m]);
            a0 = p4fma(w, p4sub(ghi, gd), a0);
            a1 = p4fma(w, p4sub(gu, glo), a1);
            lo = dn;
            hi = up;
            glo = gd;
            ghi = gu;
        }
        const float4 o0 = f4(a0), o1 = f4(a1);
        L[0][0] = o0.x;
        L[0][1] = o0.y;
        L[0][2] = o0.z;
        L[0][3] = o0.w;
        L[R - 1][0] = o1.x;
        L[R - 1][1] = o1.y;
        L[R - 1][2] = o1.z;
        L[R - 1][3] = o1.w;
    }
}

template <int R>
__device__ __forceinline__ Group decode(const StepParams2D& p, int item) {
    Group q;
    q.mi = model_of(p, item);
    const ModelStep2D& M = p.m[q.mi];
    const int r = item - M.item_begin;
    q.unit = r / M.ws_ntiles;
    q.tile = r - q.unit * M.ws_ntiles;
    const int tz = q.tile / M.tiles_x;
    q.z0 = tz * Ws<R>::TZ;
    q.x0 = (q.tile - tz * M.tiles_x) * kTX;
    q.f = 0;
    q.last = 0;
    q.inj = 0;
    q.fast = (q.z0 >= M.pad) && (q.z0 + Ws<R>::TZ <= M.pad + M.nz) && (q.x0 >= M.pad) &&
             (q.x0 + kTX <= M.pad + M.nx);
    q.rbeg = M.ws_rec_ptr[q.tile];
    q.rend = M.ws_rec_ptr[q.tile + 1];
    q.sz = q.sx = 0;
    q.fsrc = 0.f;
    return q;
}

__device__ __forceinline__ void fail_exit(int* err) { set_dev_error(err, DEVERR_TIMEOUT); }

// Receivers of the tile sampled from a staged halo tile (field at time n).
__device__ __forceinline__ void sample_recv(const float* st, const ModelStep2D& M, const Group& q, float* out,
                                            int tid) {
    for (int i = q.rbeg + tid; i < q.rend; i += kThreads) {
        const int r = M.ws_rec_idx[i];
        out[r] = st[(M.rec_zx[2 * r] - q.z0 + 4) * HX + (M.rec_zx[2 * r + 1] - q.x0 + 4)];
    }
}

// ---- forward ---------------------------------------------------------------
template <int KIND, int S, bool MULTI, int R>
__global__ void __launch_bounds__(kWsThreads, R == 1 ? 4 : 3) k_fwd2d_ws(const __grid_constant__ StepParams2D p) {
    using T = Ws<R>;
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
        int s = 0, g = 0;
        uint32_t eph = 0;  // phase of empty[s] to wait for (once the ring has wrapped)
        // the next item is decoded one item ahead, so that its global lookups (receiver range,
        // source cell, wavelet sample) overlap the waits of the current one
        auto decode_fwd = [&](int it) {
            Group d = decode<R>(p, it);
            const ModelStep2D& Md = p.m[d.mi];
            d.sz = Md.src_zx[2 * d.unit];
            d.sx = Md.src_zx[2 * d.unit + 1];
            d.fsrc = Md.wavelet[n] * Md.vol_inv;
            return d;
        };
        Group qn = (blockIdx.x < total) ? decode_fwd(blockIdx.x) : Group{};
        for (int item = blockIdx.x;; item += gridDim.x) {
            const bool done = item >= total;
            Group q = qn;
            if (!done && item + (int)gridDim.x < total) qn = decode_fwd(item + gridDim.x);
            const int ngr = done ? 1 : (KIND == FWD_BORN ? 1 + p.m[q.mi].nb : 1);
            for (int f = 0; f < ngr; ++f, ++g) {
                if (g >= S && !mbar_wait_bounded(&empty[s], eph)) {
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
                info[s] = q;
                float* st = smem + s * T::FWD_STAGE;
                mbar_expect_tx(&full[s], T::HALO_B + 2 * T::PLAIN_B);
                if (f == 0) {
                    tma_load_3d(st, &M.tm_wu, q.x0 - 4, q.z0 - 4, q.unit * 2 + pc, &full[s]);
                    tma_load_3d(st + T::HALO, &M.tm_sp, q.x0, q.z0, 0, &full[s]);
                    tma_load_3d(st + T::HALO + T::PLAIN, &M.tm_up, q.x0, q.z0, q.unit * 2 + po, &full[s]);
                } else {
                    const int b = f - 1;
                    const int pl = (q.unit * M.nb + b) * 2;
                    tma_load_3d(st, &M.tm_wf, q.x0 - 4, q.z0 - 4, pl + pc, &full[s]);
                    tma_load_3d(st + T::HALO, &M.tm_dmp, q.x0, q.z0, b, &full[s]);
                    tma_load_3d(st + T::HALO + T::PLAIN, &M.tm_fp, q.x0, q.z0, pl + po, &full[s]);
                }
                if (++s == S) {
                    s = 0;
                    if (g + 1 >= 2 * S) eph ^= 1u;  // the wait for group g+1 is for use (g+1)/S - 1
                }
            }
        }
    }

    // ---------------- consumer warps
    const int lx = (tid & 15) << 2, lz = (tid >> 4) * R;
    float4 sv[R];
    float D[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        sv[r] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 4; ++j) D[r][j] = 0.f;
    }
    int s = 0;
    uint32_t ph = 0;
    for (;;) {
        if (!mbar_wait_bounded(&full[s], ph)) {
            fail_exit(p.err);
            return;
        }
        const Group q = info[s];
        if (q.f < 0) return;
        const ModelStep2D& M = p.m[MULTI ? q.mi : 0];  // single model: loop-invariant descriptor
        const float* st = smem + s * T::FWD_STAGE;
        const int shot = q.unit;
        const int x = q.x0 + lx;
        const bool fast = q.fast != 0;
        float L[R][4];
        float4 c[R];
        lap_rows<R, true>(st, lz + 4, lx + 4, M, c, L);
        if (q.f == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int z = q.z0 + lz + r;
                sv[r] = ld4(st + T::HALO + (lz + r) * kTX + lx);
                const float4 pold = ld4(st + T::HALO + T::PLAIN + (lz + r) * kTX + lx);
                if (z == q.sz) add_lane(L[r], q.sx - x, q.fsrc);
                float o[4];
                if (fast) {
                    const P4 Fo = p4mul(p4(sv[r]), p4(L[r][0], L[r][1], L[r][2], L[r][3]));
                    const float4 Dv = f4(p4mul(Fo, p4(M.inv_dt2, M.inv_dt2, M.inv_dt2, M.inv_dt2)));
                    const float4 ov = f4(p4leap1(p4(c[r]), p4(pold), Fo));
                    D[r][0] = Dv.x, D[r][1] = Dv.y, D[r][2] = Dv.z, D[r][3] = Dv.w;
                    o[0] = ov.x, o[1] = ov.y, o[2] = ov.z, o[3] = ov.w;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float Fo = __fmul_rn(get(sv[r], j), L[r][j]);
                        D[r][j] = __fmul_rn(Fo, M.inv_dt2);
                        o[j] = cell_update(M, false, z, x + j, get(c[r], j), get(pold, j), Fo);
                    }
                }
                if (fast || (z < M.Nz && x < M.Nx)) {
                    const long long off = (long long)z * M.P + x;
                    st4(M.u + (long long)(shot * 2 + po) * M.F + off, make_float4(o[0], o[1], o[2], o[3]));
                    if (KIND == FWD_INCIDENT_DTT || (KIND == FWD_BORN && M.dtt_store))
                        st4(M.dtt + (long long)shot * M.dtt_shot_stride + (long long)M.dtt_slot * M.F + off,
                            make_float4(D[r][0], D[r][1], D[r][2], D[r][3]));
                }
            }
            if (KIND == FWD_INCIDENT_SAMPLE && q.rend > q.rbeg)
                sample_recv(st, M, q, M.data + (long long)shot * M.data_shot_stride + (long long)n * M.nr, tid);
        } else {
            const int b = q.f - 1;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int z = q.z0 + lz + r;
                const float4 dmv = ld4(st + T::HALO + (lz + r) * kTX + lx);
                const float4 fo = ld4(st + T::HALO + T::PLAIN + (lz + r) * kTX + lx);
                float o[4];
                if (fast) {
                    const P4 src = p4fma(p4neg(p4(dmv)), p4(D[r][0], D[r][1], D[r][2], D[r][3]),
                                         p4(L[r][0], L[r][1], L[r][2], L[r][3]));
                    const float4 ov = f4(p4leap1(p4(c[r]), p4(fo), p4mul(p4(sv[r]), src)));
                    o[0] = ov.x, o[1] = ov.y, o[2] = ov.z, o[3] = ov.w;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float src = __fmaf_rn(-get(dmv, j), D[r][j], L[r][j]);
                        o[j] = cell_update(M, false, z, x + j, get(c[r], j), get(fo, j), __fmul_rn(get(sv[r], j), src));
                    }
                }
                if (fast || (z < M.Nz && x < M.Nx))
                    st4(M.f + (long long)((shot * M.nb + b) * 2 + po) * M.F + (long long)z * M.P + x,
                        make_float4(o[0], o[1], o[2], o[3]));
            }
            if (q.rend > q.rbeg)
                sample_recv(st, M, q,
                            M.data + (long long)shot * M.data_shot_stride + (long long)b * M.data_trial_stride +
                                (long long)n * M.nr,
                            tid);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == S) {
            s = 0;
            ph ^= 1u;
        }
    }
}

// ---- adjoint ---------------------------------------------------------------
// Item = (model, shot group, tile); its groups are (shot jj of the group, trial bi of the chunk),
// jj-major.  s is staged with the item's first group, Dtt with each shot's first trial.
template <int NBC, bool KAHAN, int S, bool MULTI, int R>
__global__ void __launch_bounds__(kWsThreads, (NBC * R >= 8) ? 1 : 2) k_adj2d_ws(const __grid_constant__ StepParams2D p) {
    using T = Ws<R>;
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
        int s = 0, g = 0;
        uint32_t eph = 0;
        Group qn = (blockIdx.x < total) ? decode<R>(p, blockIdx.x) : Group{};  // one item ahead
        for (int item = blockIdx.x;; item += gridDim.x) {
            const bool done = item >= total;
            Group q = qn;
            if (!done && item + (int)gridDim.x < total) qn = decode<R>(p, item + gridDim.x);
            int nsh = 1, nbc = 1;
            if (!done) {
                const ModelStep2D& M = p.m[q.mi];
                nsh = min(M.shot_group, M.nshots - q.unit * M.shot_group);
                nbc = min(NBC, M.nb - M.chunk * NBC);
            }
            for (int jj = 0; jj < nsh; ++jj) {
                for (int bi = 0; bi < nbc; ++bi, ++g) {
                    bool ok = true;
                    if (lane == 0 && g >= S) ok = mbar_wait_bounded(&empty[s], eph);
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
                    float* st = smem + s * T::ADJ_STAGE;
                    const int shot = q.unit * M.shot_group + jj;
                    const int b = M.chunk * NBC + bi;
                    const bool inj = q.rend > q.rbeg;  // the consumers add the prebuilt R^T r^n
                    if (lane == 0) {
                        Group gi = q;
                        gi.f = jj * NBC + bi;
                        gi.last = jj == nsh - 1;  // trial bi's sum over the shot group is complete here
                        gi.inj = inj;
                        info[s] = gi;
                        const int pl = (shot * M.nb + b) * 2;
                        const bool with_d = bi == 0, with_s = (jj == 0) && (bi == 0), with_i = gi.last;
                        mbar_expect_tx(&full[s], T::HALO_B + T::PLAIN_B + (with_d ? T::PLAIN_B : 0u) +
                                                     (with_s ? T::PLAIN_B : 0u) +
                                                     (with_i ? (KAHAN ? 2u : 1u) * T::PLAIN_B : 0u));
                        tma_load_3d(st, &M.tm_wf, q.x0 - 4, q.z0 - 4, pl + pc, &full[s]);
                        tma_load_3d(st + T::HALO, &M.tm_fp, q.x0, q.z0, pl + po, &full[s]);
                        if (with_d)
                            tma_load_3d(st + T::HALO + T::PLAIN, &M.tm_dtp, q.x0, q.z0,
                                        shot * M.dtt_slots + M.dtt_slot, &full[s]);
                        if (with_s) tma_load_3d(st + T::HALO + 2 * T::PLAIN, &M.tm_sp, q.x0, q.z0, 0, &full[s]);
                        if (with_i) {  // trial b's image tile (and compensation), added to at this group
                            const int ip = q.unit * M.nb + b;
                            tma_load_3d(st + T::HALO + 3 * T::PLAIN, &M.tm_img, q.x0, q.z0, ip, &full[s]);
                            if (KAHAN) tma_load_3d(st + T::HALO + 4 * T::PLAIN, &M.tm_cmp, q.x0, q.z0, ip, &full[s]);
                        }
                    }
                    __syncwarp();
                    if (++s == S) {
                        s = 0;
                        if (g + 1 >= 2 * S) eph ^= 1u;  // the wait for group g+1 is for use (g+1)/S - 1
                    }
                }
            }
        }
    }

    // ---------------- consumer warps
    const int lx = (tid & 15) << 2, lz = (tid >> 4) * R;
    float acc[NBC][R][4];
#pragma unroll
    for (int k = 0; k < NBC; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[k][r][j] = 0.f;
    float4 sv[R], Dv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) sv[r] = Dv[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    int s = 0;
    uint32_t ph = 0;
    for (;;) {
        if (!mbar_wait_bounded(&full[s], ph)) {
            fail_exit(p.err);
            return;
        }
        const Group q = info[s];
        if (q.f < 0) return;
        const ModelStep2D& M = p.m[MULTI ? q.mi : 0];  // single model: loop-invariant descriptor
        const float* st = smem + s * T::ADJ_STAGE;
        const int jj = q.f / NBC, bi = q.f - (q.f / NBC) * NBC;
        const int shot = q.unit * M.shot_group + jj;
        const int b = M.chunk * NBC + bi;
        const int x = q.x0 + lx;
        const bool fast = q.fast != 0;
        if (bi == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) Dv[r] = ld4(st + T::HALO + T::PLAIN + (lz + r) * kTX + lx);
        }
        if (q.f == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) sv[r] = ld4(st + T::HALO + 2 * T::PLAIN + (lz + r) * kTX + lx);
        }
        float L[R][4];
        float4 c[R];
        lap_rows<R, false>(st, lz + 4, lx + 4, M, c, L);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int z = q.z0 + lz + r;
            const float4 mo = ld4(st + T::HALO + (lz + r) * kTX + lx);
            if (q.inj && z < M.Nz && x < M.Nx) {  // receiver injection R^T r^n, prebuilt for the segment
                const int band = M.rrow[z];
                if (band >= 0) {
                    const float4 in = ld4(M.inj + (((long long)M.inj_slot * M.nshots + shot) * M.nb + b) *
                                                      ((long long)M.nband * M.P) + (long long)band * M.P + x);
                    L[r][0] += in.x;
                    L[r][1] += in.y;
                    L[r][2] += in.z;
                    L[r][3] += in.w;
                }
            }
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                o[j] = cell_update(M, fast, z, x + j, get(c[r], j), get(mo, j), __fmul_rn(get(sv[r], j), L[r][j]));
#pragma unroll
            for (int k = 0; k < NBC; ++k)
                if (k == bi) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[k][r][j] = fmaf(-get(Dv[r], j), o[j], acc[k][r][j]);
                }
            if (fast || (z < M.Nz && x < M.Nx))
                st4(M.f + (long long)((shot * M.nb + b) * 2 + po) * M.F + (long long)z * M.P + x,
                    make_float4(o[0], o[1], o[2], o[3]));
        }
        if (q.last) {  // trial b's sum over the shot group is complete: add it to its image tile
            float* img = M.img + (long long)q.unit * M.img_group_stride + (long long)b * M.F;
            float* cmp = M.comp + (long long)q.unit * M.img_group_stride + (long long)b * M.F;
#pragma unroll
            for (int k = 0; k < NBC; ++k)
                if (k == bi) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int z = q.z0 + lz + r;
                        if (fast || (z < M.Nz && x < M.Nx)) {
                            const long long off = (long long)z * M.P + x;
                            const float* ist = st + T::HALO + 3 * T::PLAIN + (lz + r) * kTX + lx;
                            float4 iv = ld4(ist);
                            if (KAHAN) {
                                float4 cv = ld4(ist + T::PLAIN);
                                kahan4(iv, cv, acc[k][r][0], acc[k][r][1], acc[k][r][2], acc[k][r][3]);
                                st4(cmp + off, cv);
                            } else {
                                iv.x += acc[k][r][0];
                                iv.y += acc[k][r][1];
                                iv.z += acc[k][r][2];
                                iv.w += acc[k][r][3];
                            }
                            st4(img + off, iv);
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[k][r][j] = 0.f;
                    }
                }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == S) {
            s = 0;
            ph ^= 1u;
        }
    }
}

int occupancy(const void* fn, size_t smem) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kWsThreads, smem);
    return nb < 1 ? 1 : nb;
}

int num_sms() {
    static const int n = [] {  // initialised once, thread-safe (function-local static)
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v < 1 ? 1 : v;
    }();
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

template <int R>
size_t smem_bytes(int stages, bool adjoint) {
    return (size_t)stages * (adjoint ? Ws<R>::ADJ_STAGE : Ws<R>::FWD_STAGE) * 4;
}

template <int K, int R>
cudaError_t launch_fwd_kr(int stages, const StepParams2D& p, cudaStream_t st) {
    const size_t sm = smem_bytes<R>(stages, false);
    const int total = p.total_items;
    if (p.nmodels > 1)
        return stages == 3 ? launch_persistent(k_fwd2d_ws<K, 3, true, R>, sm, total, p, st)
                           : launch_persistent(k_fwd2d_ws<K, 2, true, R>, sm, total, p, st);
    return stages == 3 ? launch_persistent(k_fwd2d_ws<K, 3, false, R>, sm, total, p, st)
                       : launch_persistent(k_fwd2d_ws<K, 2, false, R>, sm, total, p, st);
}

template <int NB, bool KH, int R>
cudaError_t launch_adj_nkr(int stages, const StepParams2D& q, cudaStream_t st) {
    const size_t sm = smem_bytes<R>(stages, true);
    const int total = q.total_items;
    if (q.nmodels > 1)
        return stages == 3 ? launch_persistent(k_adj2d_ws<NB, KH, 3, true, R>, sm, total, q, st)
                           : launch_persistent(k_adj2d_ws<NB, KH, 2, true, R>, sm, total, q, st);
    return stages == 3 ? launch_persistent(k_adj2d_ws<NB, KH, 3, false, R>, sm, total, q, st)
                       : launch_persistent(k_adj2d_ws<NB, KH, 2, false, R>, sm, total, q, st);
}

template <int NB, bool KH>
cudaError_t launch_adj_nk(int stages, const StepParams2D& q, cudaStream_t st) {
    return q.m[0].ws_rows == 2 ? launch_adj_nkr<NB, KH, 2>(stages, q, st) : launch_adj_nkr<NB, KH, 1>(stages, q, st);
}

}  // namespace

size_t pipe_smem_bytes(int stages, bool adjoint, int rows) {
    return rows == 2 ? smem_bytes<2>(stages, adjoint) : smem_bytes<1>(stages, adjoint);
}

// stages: 2 or 3 (anything else runs 2); the tile height is 16 * p.m[0].ws_rows (same for all models).
cudaError_t launch_fwd2d_pipe(FwdKind kind, int stages, const StepParams2D& p, cudaStream_t st) {
    if (p.total_items <= 0) return cudaSuccess;
    const bool r2 = p.m[0].ws_rows == 2;
    switch (kind) {
        case FWD_INCIDENT:
            return r2 ? launch_fwd_kr<FWD_INCIDENT, 2>(stages, p, st) : launch_fwd_kr<FWD_INCIDENT, 1>(stages, p, st);
        case FWD_INCIDENT_DTT:
            return r2 ? launch_fwd_kr<FWD_INCIDENT_DTT, 2>(stages, p, st)
                      : launch_fwd_kr<FWD_INCIDENT_DTT, 1>(stages, p, st);
        case FWD_BORN:
            return r2 ? launch_fwd_kr<FWD_BORN, 2>(stages, p, st) : launch_fwd_kr<FWD_BORN, 1>(stages, p, st);
        case FWD_INCIDENT_SAMPLE:
            return r2 ? launch_fwd_kr<FWD_INCIDENT_SAMPLE, 2>(stages, p, st)
                      : launch_fwd_kr<FWD_INCIDENT_SAMPLE, 1>(stages, p, st);
    }
    return cudaErrorInvalidValue;
}

// nbc: trials per CTA (1, 2, 4 or 8; at most 4 with two rows per thread).
cudaError_t launch_adj2d_pipe(int nbc, bool kahan, int stages, const StepParams2D& p, int chunks, cudaStream_t st) {
    if (p.total_items <= 0) return cudaSuccess;
    if (nbc == 8 && p.m[0].ws_rows == 2) return cudaErrorInvalidValue;
    StepParams2D q = p;
    for (int c = 0; c < chunks; ++c) {
        for (int k = 0; k < q.nmodels; ++k) q.m[k].chunk = c;
        cudaError_t e;
        switch (nbc) {
            case 1: e = kahan ? launch_adj_nk<1, true>(stages, q, st) : launch_adj_nk<1, false>(stages, q, st); break;
            case 2: e = kahan ? launch_adj_nk<2, true>(stages, q, st) : launch_adj_nk<2, false>(stages, q, st); break;
            case 4: e = kahan ? launch_adj_nk<4, true>(stages, q, st) : launch_adj_nk<4, false>(stages, q, st); break;
            case 8:
                e = kahan ? launch_adj_nkr<8, true, 1>(stages, q, st) : launch_adj_nkr<8, false, 1>(stages, q, st);
                break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace probe
