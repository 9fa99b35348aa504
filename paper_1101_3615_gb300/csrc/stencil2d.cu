// 2D time-stepping kernels of the Born / migration sweeps (sm_103a).
//
// One launch advances every resident (model, shot) by one time step.  A CTA of
// 256 threads owns a 64 x TZ tile of one shot; the radius-4 halo tile of the
// field being differentiated is staged in shared memory by a TMA tiled load
// (cp.async.bulk.tensor, zero fill outside the padded grid = the zero
// extension of the Laplacian), the pointwise operands (previous level, s, dm,
// Dtt u) stream through coalesced float4 loads, and each thread updates 4
// consecutive x cells per row.  The sponge factors are computed from the cell
// index, the point source and the receivers are handled inside the tile.
//
// Scheme (Sec. 2 wave equations, 2nd order in time / 8th order in space):
//   u^{n+1}  = G [2u^n  - a- u^{n-1}  + s (L u^n + f^n)]
//   du^{n+1} = G [2du^n - a- du^{n-1} + s (L du^n - dm Dtt u^n)],
//   Dtt u^n  = s (L u^n + f^n) / dt^2   (exact in the interior, where dm lives)
// Adjoint (exact transpose, written for the scaled variable mu = s G lambda,
// which obeys the same recurrence run backwards in time):
//   mu^n = G [2mu^{n+1} - a- mu^{n+2} + s (L mu^{n+1} + R^T r^n)]
//   img -= Dtt u^{n-1} * mu^n                 (zero-lag imaging, Sec. 1.1 RTM)
#include "common.cuh"
#include "internal.h"

namespace probe {

template <int TZ>
struct Tile2D {
    static constexpr int HX = kTX + 8;
    static constexpr int HZ = TZ + 8;
    static constexpr int FLOATS = HX * HZ;
    static constexpr unsigned BYTES = FLOATS * 4u;
    static constexpr int ROWS = TZ / 16;
};

// Grid: x = tile column, y = tile row, z = (model, shot or shot group) linearised
// over the models of the launch; CTAs beyond a smaller model's tile range exit.
__device__ __forceinline__ int find_model(const StepParams2D& p, int bz) {
    int mi = 0;
#pragma unroll
    for (int k = 1; k < kMaxModels; ++k)
        if (k < p.nmodels && bz >= p.m[k].block_begin) mi = k;
    return mi;
}

// Laplacian of the 4 cells starting at tile coordinates (row, col) (col % 4 == 0).
// The taps are accumulated from differences of neighbouring values, never from
// the raw values against the centre term: those differences are nearly exact in
// FP32, which removes the cancellation that otherwise dominates the round-off
// of the time stepping for smooth, well-sampled fields.  Per axis, with
// d_i = v_{i+1} - v_i,
//   sum_k w_k (v_{c+k} + v_{c-k} - 2 v_c) = sum_{m=0..3} C_m (d_{c+m} - d_{c-m-1}),
//   C_m = sum_{k>m} w_k / h^2;
// x first (11 shared differences for the thread's 4 cells), then z (8 per
// column).  The pipelined kernels evaluate the same operations in the same
// order, so both families give the same bits.
template <int HX>
__device__ __forceinline__ void lap4(const float* t, int row, int col, const ModelStep2D& M,
                                     float4& center, float L[4]) {
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
    // z, outward from the centre row: the term m pairs d_{3-m} = v_{4-m} - v_{3-m} below
    // with d_{4+m} = v_{5+m} - v_{4+m} above (v_4 = b), so few rows are live at once.
    float4 lo = b, hi = b;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float4 dn = ld4(rp - (m + 1) * HX), up = ld4(rp + (m + 1) * HX);
        L[0] = fmaf(M.czm[m], (up.x - hi.x) - (lo.x - dn.x), L[0]);
        L[1] = fmaf(M.czm[m], (up.y - hi.y) - (lo.y - dn.y), L[1]);
        L[2] = fmaf(M.czm[m], (up.z - hi.z) - (lo.z - dn.z), L[2]);
        L[3] = fmaf(M.czm[m], (up.w - hi.w) - (lo.w - dn.w), L[3]);
        lo = dn;
        hi = up;
    }
}

// Sponge term e = eta dt / 2 of a padded cell (zero in the interior).
__device__ __forceinline__ float sponge_e(const ModelStep2D& M, int z, int x) {
    const int rz = max(max(M.pad - z, z - (M.pad + M.nz - 1)), 0);
    const int rx = max(max(M.pad - x, x - (M.pad + M.nx - 1)), 0);
    return __fmaf_rn(M.cz, (float)(rz * rz), __fmul_rn(M.cx, (float)(rx * rx)));
}

// G = 1/(1 + e) and a- = 1 - e of a sponge cell (left at 1 where e = 0).
__device__ __forceinline__ void sponge_factors(const ModelStep2D& M, int z, int x, float& G, float& am) {
    sponge_pair(sponge_e(M, z, x), G, am);
}

// Record the receivers of this tile from a staged field tile.
template <int HX>
__device__ __forceinline__ void sample_tile(const float* t, const ModelStep2D& M, int tile, int z0,
                                            int x0, float* out) {
    const int beg = M.rec_tile_ptr[tile], end = M.rec_tile_ptr[tile + 1];
    for (int i = beg + (int)threadIdx.x; i < end; i += kThreads) {
        const int r = M.rec_tile_idx[i];
        const int rz = M.rec_zx[2 * r], rx = M.rec_zx[2 * r + 1];
        out[r] = t[(rz - z0 + 4) * HX + (rx - x0 + 4)];
    }
}

// After a failed bounded wait: flag the error and give the copies in flight
// one more bounded wait before the CTA releases its shared memory.
__device__ __forceinline__ void abort_cta(int* err, uint64_t* bars, int nbars,
                                          const uint32_t* parity) {
    if (threadIdx.x == 0) {
        set_dev_error(err, DEVERR_TIMEOUT);
        for (int i = 0; i < nbars; ++i) (void)mbar_wait_bounded(&bars[i], parity[i]);
    }
}

template <int TZ, int KIND>
__global__ void __launch_bounds__(kThreads, TZ == 16 ? 4 : 3) k_fwd2d(const __grid_constant__ StepParams2D p) {
    using T = Tile2D<TZ>;
    constexpr int HX = T::HX;
    constexpr int ROWS = T::ROWS;
    constexpr bool BORN = (KIND == FWD_BORN);
    constexpr bool DTT = (KIND == FWD_INCIDENT_DTT);
    constexpr bool SAMPLE_U = (KIND == FWD_INCIDENT_SAMPLE);

    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[3];

    const int mi = find_model(p, blockIdx.z);
    const ModelStep2D& M = p.m[mi];
    if ((int)blockIdx.x >= M.tiles_x || (int)blockIdx.y >= M.tiles_z) return;
    const int shot = blockIdx.z - M.block_begin;
    const int tile = blockIdx.y * M.tiles_x + blockIdx.x;
    const int z0 = blockIdx.y * TZ, x0 = blockIdx.x * kTX;
    const int tid = threadIdx.x;
    const int lx = (tid & 15) << 2, lz = tid >> 4;
    const int n = p.n;
    const int pc = n & 1, po = pc ^ 1;
    const long long F = M.F;
    float* su = smem;
    float* sf0 = smem + T::FLOATS;
    float* sf1 = smem + 2 * T::FLOATS;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&bars[0], T::BYTES);
        tma_load_3d(su, &M.tm_u, x0 - 4, z0 - 4, shot * 2 + pc, &bars[0]);
        if (BORN && M.nb > 0) {
            mbar_expect_tx(&bars[1], T::BYTES);
            tma_load_3d(sf0, &M.tm_f, x0 - 4, z0 - 4, (shot * M.nb) * 2 + pc, &bars[1]);
        }
    }

    const int x = x0 + lx;
    const bool full = (x0 + kTX <= M.Nx);  // no pitch column inside this tile
    float* ubase = M.u + (long long)(shot * 2) * F;
    float4 sv[ROWS], uo[ROWS];
    long long off[ROWS];
    bool valid[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int z = z0 + lz + 16 * r;
        valid[r] = (z < M.Nz) && (x < M.Nx);
        off[r] = (long long)z * M.P + x;
        sv[r] = valid[r] ? ld4(M.s + off[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
        uo[r] = valid[r] ? ld4(ubase + po * F + off[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }

    const uint32_t par0[3] = {0u, 0u, 0u};
    const bool ok0 = mbar_wait_bounded(&bars[0], 0);
    if (__syncthreads_or(!ok0)) {
        abort_cta(p.err, bars, BORN && M.nb > 0 ? 2 : 1, par0);
        return;
    }

    const int sz = M.src_zx[2 * shot], sx = M.src_zx[2 * shot + 1];
    const float fsrc = M.wavelet[n] * M.vol_inv;
    float D[ROWS][4];
    bool interior[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int z = z0 + lz + 16 * r;
        float L[4];
        float4 c;
        lap4<HX>(su, lz + 16 * r + 4, lx + 4, M, c, L);
        if (z == sz) {
            const int j = sx - x;
            add_lane(L, j, fsrc);
        }
        float o[4];
        interior[r] = (z >= M.pad) && (z < M.pad + M.nz) && (x >= M.pad) && (x + 3 < M.pad + M.nx);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float Fo = __fmul_rn(get(sv[r], j), L[j]);
            D[r][j] = __fmul_rn(Fo, M.inv_dt2);
            float G = 1.f, am = 1.f;
            if (!interior[r]) sponge_factors(M, z, x + j, G, am);
            o[j] = (full || x + j < M.Nx) ? leapfrog(G, get(c, j), am, get(uo[r], j), Fo) : 0.f;
        }
        if (valid[r]) {
            st4(ubase + po * F + off[r], make_float4(o[0], o[1], o[2], o[3]));
            if (DTT || (BORN && M.dtt_store))
                st4(M.dtt + (long long)shot * M.dtt_shot_stride + (long long)M.dtt_slot * F + off[r],
                    make_float4(D[r][0], D[r][1], D[r][2], D[r][3]));
        }
    }
    if (SAMPLE_U)
        sample_tile<HX>(su, M, tile, z0, x0, M.data + (long long)shot * M.data_shot_stride +
                                                 (long long)n * M.nr);

    if (BORN) {
        const int nb = M.nb;
        for (int b = 0; b < nb; ++b) {
            const int buf = b & 1;
            float* sf = buf ? sf1 : sf0;
            if (tid == 0 && b + 1 < nb) {
                mbar_expect_tx(&bars[1 + (buf ^ 1)], T::BYTES);
                tma_load_3d(buf ? sf0 : sf1, &M.tm_f, x0 - 4, z0 - 4, ((shot * nb + b + 1) * 2) + pc,
                            &bars[1 + (buf ^ 1)]);
            }
            float* fb = M.f + (long long)((shot * nb + b) * 2) * F;
            const float* dmb = M.dm + (long long)b * F;
            float4 dv[ROWS], fo[ROWS];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                dv[r] = valid[r] ? ld4(dmb + off[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
                fo[r] = valid[r] ? ld4(fb + po * F + off[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const bool ok = mbar_wait_bounded(&bars[1 + buf], (b >> 1) & 1);
            if (__syncthreads_or(!ok)) {
                const uint32_t par[3] = {0u, (uint32_t)((b >> 1) & 1), (uint32_t)((b >> 1) & 1)};
                abort_cta(p.err, bars + 1 + buf, 1, par + 1 + buf);
                return;
            }
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                float L[4];
                float4 c;
                lap4<HX>(sf, lz + 16 * r + 4, lx + 4, M, c, L);
                float o[4];
                const int z = z0 + lz + 16 * r;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float src = __fmaf_rn(-get(dv[r], j), D[r][j], L[j]);
                    float G = 1.f, am = 1.f;
                    if (!interior[r]) sponge_factors(M, z, x + j, G, am);
                    o[j] = (full || x + j < M.Nx)
                               ? leapfrog(G, get(c, j), am, get(fo[r], j), __fmul_rn(get(sv[r], j), src))
                               : 0.f;
                }
                if (valid[r]) st4(fb + po * F + off[r], make_float4(o[0], o[1], o[2], o[3]));
            }
            sample_tile<HX>(sf, M, tile, z0, x0,
                            M.data + (long long)shot * M.data_shot_stride +
                                (long long)b * M.data_trial_stride + (long long)n * M.nr);
            __syncthreads();
        }
    }
}

template <int TZ, int NBC, bool KAHAN>
__global__ void __launch_bounds__(kThreads, (NBC * TZ <= 32) ? 4 : 2) k_adj2d(const __grid_constant__ StepParams2D p) {
    using T = Tile2D<TZ>;
    constexpr int HX = T::HX;
    constexpr int ROWS = T::ROWS;

    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bars[2];

    const int mi = find_model(p, blockIdx.z);
    const ModelStep2D& M = p.m[mi];
    if ((int)blockIdx.x >= M.tiles_x || (int)blockIdx.y >= M.tiles_z) return;
    const int grp = blockIdx.z - M.block_begin;
    const int tile = blockIdx.y * M.tiles_x + blockIdx.x;
    const int z0 = blockIdx.y * TZ, x0 = blockIdx.x * kTX;
    const int tid = threadIdx.x;
    const int lx = (tid & 15) << 2, lz = tid >> 4;
    const int n = p.n;
    const int pc = (n + 1) & 1;  // plane of mu^{n+1}
    const int po = n & 1;        // plane of mu^{n+2}, overwritten by mu^n
    const long long F = M.F;
    const int nb = M.nb;
    const int b0 = M.chunk * NBC;
    if (b0 >= nb) return;
    const int nbc = min(NBC, nb - b0);
    const int j0 = grp * M.shot_group;
    const int nsh = min(M.shot_group, M.nshots - j0);
    const int niter = nsh * nbc;
    float* sbuf[2] = {smem, smem + T::FLOATS};

    const int rbeg = M.rec_tile_ptr[tile], rend = M.rec_tile_ptr[tile + 1];
    const bool has_rec = rend > rbeg;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0 && niter > 0) {
        mbar_expect_tx(&bars[0], T::BYTES);
        tma_load_3d(sbuf[0], &M.tm_f, x0 - 4, z0 - 4, ((j0 * nb + b0) * 2) + pc, &bars[0]);
    }

    const int x = x0 + lx;
    const bool full = (x0 + kTX <= M.Nx);
    float4 sv[ROWS];
    long long off[ROWS];
    bool valid[ROWS], interior[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int z = z0 + lz + 16 * r;
        valid[r] = (z < M.Nz) && (x < M.Nx);
        off[r] = (long long)z * M.P + x;
        sv[r] = valid[r] ? ld4(M.s + off[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
        interior[r] = (z >= M.pad) && (z < M.pad + M.nz) && (x >= M.pad) && (x + 3 < M.pad + M.nx);
    }

    float acc[NBC][ROWS][4];
#pragma unroll
    for (int bi = 0; bi < NBC; ++bi)
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[bi][r][j] = 0.f;

    for (int jj = 0; jj < nsh; ++jj) {
        const int shot = j0 + jj;
        float4 Dv[ROWS];
        const float* dtt = M.dtt + (long long)shot * M.dtt_shot_stride + (long long)M.dtt_slot * F;
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
            Dv[r] = valid[r] ? ld4(dtt + off[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int bi = 0; bi < NBC; ++bi) {
            if (bi < nbc) {
                const int it = jj * nbc + bi;
                const int buf = it & 1;
                const int b = b0 + bi;
                if (tid == 0 && it + 1 < niter) {
                    const int jn = j0 + (it + 1) / nbc, bn = b0 + (it + 1) % nbc;
                    mbar_expect_tx(&bars[buf ^ 1], T::BYTES);
                    tma_load_3d(sbuf[buf ^ 1], &M.tm_f, x0 - 4, z0 - 4, ((jn * nb + bn) * 2) + pc,
                                &bars[buf ^ 1]);
                }
                // operands of the next iteration (its mu^{n+2}, a new shot's Dtt) or, on the last
                // one, the image tiles: into L2 while this iteration computes
                if (it + 1 < niter) {
                    const int jn = j0 + (it + 1) / nbc, bn = b0 + (it + 1) % nbc;
                    const float* fn = M.f + (long long)((jn * nb + bn) * 2 + po) * F;
                    const float* dn = M.dtt + (long long)jn * M.dtt_shot_stride + (long long)M.dtt_slot * F;
#pragma unroll
                    for (int r = 0; r < ROWS; ++r) {
                        if (!valid[r]) continue;
                        prefetch_l2(fn + off[r]);
                        if ((it + 1) % nbc == 0) prefetch_l2(dn + off[r]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < NBC; ++k) {
                        if (k >= nbc) continue;
                        const long long boff = (long long)grp * M.img_group_stride + (long long)(b0 + k) * F;
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) {
                            if (!valid[r]) continue;
                            prefetch_l2(M.img + boff + off[r]);
                            if (KAHAN) prefetch_l2(M.comp + boff + off[r]);
                        }
                    }
                }
                float* fb = M.f + (long long)((shot * nb + b) * 2) * F;
                float4 mo[ROWS], inj[ROWS];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    mo[r] = valid[r] ? ld4(fb + po * F + off[r]) : make_float4(0.f, 0.f, 0.f, 0.f);
                    // receiver injection R^T r^n, prebuilt for this segment (rows with receivers only)
                    inj[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (has_rec && valid[r]) {
                        const int band = M.rrow[z0 + lz + 16 * r];
                        if (band >= 0)
                            inj[r] = ld4(M.inj + (((long long)M.inj_slot * M.nshots + shot) * nb + b) *
                                                     ((long long)M.nband * M.P) + (long long)band * M.P + x);
                    }
                }
                const bool ok = mbar_wait_bounded(&bars[buf], (it >> 1) & 1);
                if (__syncthreads_or(!ok)) {
                    const uint32_t par = (uint32_t)((it >> 1) & 1);
                    abort_cta(p.err, &bars[buf], 1, &par);
                    return;
                }
                const float* sf = sbuf[buf];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    float L[4];
                    float4 c;
                    lap4<HX>(sf, lz + 16 * r + 4, lx + 4, M, c, L);
                    if (has_rec) {
                        L[0] += inj[r].x;
                        L[1] += inj[r].y;
                        L[2] += inj[r].z;
                        L[3] += inj[r].w;
                    }
                    float o[4];
                    const int z = z0 + lz + 16 * r;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float G = 1.f, am = 1.f;
                        if (!interior[r]) sponge_factors(M, z, x + j, G, am);
                        o[j] = (full || x + j < M.Nx) ? leapfrog(G, get(c, j), am, get(mo[r], j), __fmul_rn(get(sv[r], j), L[j]))
                                                      : 0.f;
                        acc[bi][r][j] = fmaf(-get(Dv[r], j), o[j], acc[bi][r][j]);
                    }
                    if (valid[r]) st4(fb + po * F + off[r], make_float4(o[0], o[1], o[2], o[3]));
                }
                __syncthreads();
            }
        }
    }

    float* img = M.img + (long long)grp * M.img_group_stride;
    float* cmp = M.comp + (long long)grp * M.img_group_stride;
#pragma unroll
    for (int bi = 0; bi < NBC; ++bi) {
        if (bi < nbc) {
            const long long boff = (long long)(b0 + bi) * F;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                if (!valid[r]) continue;
                float* ip = img + boff + off[r];
                float4 iv = ld4(ip);
                if (KAHAN) {
                    float* cp = cmp + boff + off[r];
                    float4 cv = ld4(cp);
                    kahan4(iv, cv, acc[bi][r][0], acc[bi][r][1], acc[bi][r][2], acc[bi][r][3]);
                    st4(cp, cv);
                } else {
                    iv.x += acc[bi][r][0];
                    iv.y += acc[bi][r][1];
                    iv.z += acc[bi][r][2];
                    iv.w += acc[bi][r][3];
                }
                st4(ip, iv);
            }
        }
    }
}

size_t fwd2d_smem_bytes(FwdKind kind, int tile_z) {
    const size_t tile = (size_t)(kTX + 8) * (tile_z + 8) * 4;
    return kind == FWD_BORN ? 3 * tile : tile;
}

size_t adj2d_smem_bytes(int tile_z) {
    const size_t tile = (size_t)(kTX + 8) * (tile_z + 8) * 4;
    return 2 * tile;  // double-buffered halo tiles
}

template <int TZ>
static cudaError_t launch_fwd_tz(FwdKind kind, const StepParams2D& p, dim3 grid, cudaStream_t st) {
    const size_t sm = fwd2d_smem_bytes(kind, TZ);
    switch (kind) {
        case FWD_INCIDENT: k_fwd2d<TZ, FWD_INCIDENT><<<grid, kThreads, sm, st>>>(p); break;
        case FWD_INCIDENT_DTT: k_fwd2d<TZ, FWD_INCIDENT_DTT><<<grid, kThreads, sm, st>>>(p); break;
        case FWD_BORN: k_fwd2d<TZ, FWD_BORN><<<grid, kThreads, sm, st>>>(p); break;
        case FWD_INCIDENT_SAMPLE:
            k_fwd2d<TZ, FWD_INCIDENT_SAMPLE><<<grid, kThreads, sm, st>>>(p);
            break;
    }
    return cudaGetLastError();
}

static dim3 grid2d(const StepParams2D& p, int zblocks) {
    int tx = 0, tz = 0;
    for (int k = 0; k < p.nmodels; ++k) {
        tx = max(tx, p.m[k].tiles_x);
        tz = max(tz, p.m[k].tiles_z);
    }
    return dim3(tx, tz, zblocks);
}

cudaError_t launch_fwd2d(FwdKind kind, int tile_z, const StepParams2D& p, int zblocks,
                         cudaStream_t st) {
    if (zblocks <= 0) return cudaSuccess;
    const dim3 grid = grid2d(p, zblocks);
    if (tile_z == 16) return launch_fwd_tz<16>(kind, p, grid, st);
    if (tile_z == 32) return launch_fwd_tz<32>(kind, p, grid, st);
    return cudaErrorInvalidValue;
}

template <int TZ, int NBC>
static cudaError_t launch_adj_nbc(bool kahan, const StepParams2D& p, int zblocks, int chunks,
                                  cudaStream_t st) {
    const size_t sm = adj2d_smem_bytes(TZ);
    const dim3 grid = grid2d(p, zblocks);
    // trial chunks run as separate launches of the same step (each writes its own trials)
    StepParams2D q = p;
    for (int c = 0; c < chunks; ++c) {
        for (int k = 0; k < q.nmodels; ++k) q.m[k].chunk = c;
        if (kahan)
            k_adj2d<TZ, NBC, true><<<grid, kThreads, sm, st>>>(q);
        else
            k_adj2d<TZ, NBC, false><<<grid, kThreads, sm, st>>>(q);
    }
    return cudaGetLastError();
}

template <int TZ>
static cudaError_t launch_adj_tz(int nbc, bool kahan, const StepParams2D& p, int blocks, int chunks,
                                 cudaStream_t st) {
    switch (nbc) {
        case 1: return launch_adj_nbc<TZ, 1>(kahan, p, blocks, chunks, st);
        case 2: return launch_adj_nbc<TZ, 2>(kahan, p, blocks, chunks, st);
        case 4: return launch_adj_nbc<TZ, 4>(kahan, p, blocks, chunks, st);
        case 8: return launch_adj_nbc<TZ, 8>(kahan, p, blocks, chunks, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_adj2d(int tile_z, int nbc, bool kahan, const StepParams2D& p, int blocks,
                         int chunks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    if (tile_z == 16) return launch_adj_tz<16>(nbc, kahan, p, blocks, chunks, st);
    if (tile_z == 32) return launch_adj_tz<32>(nbc, kahan, p, blocks, chunks, st);
    return cudaErrorInvalidValue;
}

cudaError_t stencil2d_configure() { return cudaSuccess; }

}  // namespace probe
