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

// ---------------------------------------------------------------------------
// Time-blocked forward step: two time levels per launch (n -> n + 2), one 64 x 16 tile per CTA.
//
// The second level of a 64 x 16 output tile depends on the first level on the tile plus the
// Laplacian's radius-4 halo (the extended region E, 72 x 24), which depends on level n on the
// tile plus an 8-cell halo (80 x 32).  A CTA stages u^n (80 x 32), u^{n-1}, s (E) by TMA, computes
// u^{n+1} and Dtt u^n on all of E into shared memory (cells outside the padded grid are zero, the
// Laplacian's zero extension), then u^{n+2} on the tile; per Born trial the same with du^n,
// du^{n-1}, dm, using Dtt u^n on E and Dtt u^{n+1} on the tile.  The halo cells of E are
// recomputed by the neighbouring CTAs: 1.69x the arithmetic of the first level for half the state
// traffic -- per cell and two steps the kernel reads u^n, u^{n-1}, s and per trial du^n, du^{n-1},
// dm, and writes u^{n+1}, u^{n+2} and per trial du^{n+1}, du^{n+2}: (20 + 20 nb) bytes instead of
// the (32 + 32 nb) of two single steps.  The states hold four levels (level n in plane n & 3) so
// that no launch overwrites a level that a neighbouring tile still reads.  Every cell update is
// the one-step kernel's arithmetic (lap4, the explicit roundings of leapfrog, the same source and
// sponge terms), so both give the same bits; the receivers sample du^n and du^{n+1}.
// ---------------------------------------------------------------------------
constexpr int kTbHX = kTX + 16;       // 80
constexpr int kTbHZ = 16 + 16;        // 32
constexpr int kTbEX = kTX + 8;        // 72
constexpr int kTbEZ = 16 + 8;         // 24
constexpr int kTbH = kTbHX * kTbHZ;   // 2560 floats
constexpr int kTbE = kTbEX * kTbEZ;   // 1728 floats
constexpr int kTbGroups = (kTbEX / 4) * kTbEZ;  // 432 groups of 4 cells in E
constexpr unsigned kTbLoadBytes = (kTbH + 2 * kTbE) * 4u;

size_t fwd2d_tb_smem_bytes() { return (size_t)(2 * kTbH + 7 * kTbE) * 4; }

// One step of the incident field on 4 cells (z, x..x+3): returns u^{n+1} in o and Dtt u^n in d.
__device__ __forceinline__ void tb_incident4(const ModelStep2D& M, const float4& c, float L[4], const float4& sv,
                                             const float4& uo, int z, int x, bool store_ok, int sz, int sx, float fsrc,
                                             float o[4], float d[4]) {
    if (z == sz) add_lane(L, sx - x, fsrc);
    const bool interior = (z >= M.pad) && (z < M.pad + M.nz) && (x >= M.pad) && (x + 3 < M.pad + M.nx);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float Fo = __fmul_rn(get(sv, j), L[j]);
        d[j] = __fmul_rn(Fo, M.inv_dt2);
        float G = 1.f, am = 1.f;
        if (!interior) sponge_factors(M, z, x + j, G, am);
        o[j] = (store_ok && x + j >= 0 && x + j < M.Nx) ? leapfrog(G, get(c, j), am, get(uo, j), Fo) : 0.f;
    }
}

// One step of a Born field on 4 cells, given Dtt u^n of the cells.
__device__ __forceinline__ void tb_born4(const ModelStep2D& M, const float4& c, const float L[4], const float4& sv,
                                         const float4& fo, const float4& dv, const float d[4], int z, int x,
                                         bool store_ok, float o[4]) {
    const bool interior = (z >= M.pad) && (z < M.pad + M.nz) && (x >= M.pad) && (x + 3 < M.pad + M.nx);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float src = __fmaf_rn(-get(dv, j), d[j], L[j]);
        float G = 1.f, am = 1.f;
        if (!interior) sponge_factors(M, z, x + j, G, am);
        o[j] = (store_ok && x + j >= 0 && x + j < M.Nx) ? leapfrog(G, get(c, j), am, get(fo, j), __fmul_rn(get(sv, j), src))
                                                         : 0.f;
    }
}

// Receivers of the tile from a staged field array whose tile origin sits at (off, off).
template <int HX>
__device__ __forceinline__ void tb_sample(const float* t, int off, const ModelStep2D& M, int tile, int z0, int x0,
                                          float* out) {
    const int beg = M.rec_tile_ptr[tile], end = M.rec_tile_ptr[tile + 1];
    for (int i = beg + (int)threadIdx.x; i < end; i += kThreads) {
        const int r = M.rec_tile_idx[i];
        out[r] = t[(M.rec_zx[2 * r] - z0 + off) * HX + (M.rec_zx[2 * r + 1] - x0 + off)];
    }
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, 3) k_fwd2d_tb(const __grid_constant__ StepParams2D p) {
    constexpr bool BORN = (KIND == FWD_BORN);
    constexpr bool DTT = (KIND == FWD_INCIDENT_DTT);
    extern __shared__ __align__(128) float smem[];
    float* U0 = smem;          // u^n, tile + 8
    float* F0 = U0 + kTbH;     // du^n, tile + 8
    float* U1 = F0 + kTbH;     // u^{n-1} on E
    float* S = U1 + kTbE;      // s on E
    float* UN = S + kTbE;      // u^{n+1} on E
    float* DN = UN + kTbE;     // Dtt u^n on E
    float* F1 = DN + kTbE;     // du^{n-1} on E
    float* DM = F1 + kTbE;     // dm on E
    float* FN = DM + kTbE;     // du^{n+1} on E
    __shared__ __align__(8) uint64_t bars[2];

    const int mi = find_model(p, blockIdx.z);
    const ModelStep2D& M = p.m[mi];
    if ((int)blockIdx.x >= M.tiles_x || (int)blockIdx.y >= M.tiles_z) return;
    const int shot = blockIdx.z - M.block_begin;
    const int tile = blockIdx.y * M.tiles_x + blockIdx.x;
    const int z0 = blockIdx.y * 16, x0 = blockIdx.x * kTX;
    const int tid = threadIdx.x;
    const int n = p.n;
    const bool two = p.two != 0;
    const int pn = n & 3, pm = (n + 3) & 3, p1 = (n + 1) & 3, p2 = (n + 2) & 3;
    const long long F = M.F;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&bars[0], kTbLoadBytes);
        tma_load_3d(U0, &M.tm_u4h, x0 - 8, z0 - 8, shot * 4 + pn, &bars[0]);
        tma_load_3d(U1, &M.tm_u4e, x0 - 4, z0 - 4, shot * 4 + pm, &bars[0]);
        tma_load_3d(S, &M.tm_se, x0 - 4, z0 - 4, 0, &bars[0]);
    }
    const bool ok0 = mbar_wait_bounded(&bars[0], 0);
    if (__syncthreads_or(!ok0)) {
        const uint32_t par[1] = {0u};
        abort_cta(p.err, bars, 1, par);
        return;
    }
    const int sz = M.src_zx[2 * shot], sx = M.src_zx[2 * shot + 1];
    const float fsrc0 = M.wavelet[n] * M.vol_inv;
    const float fsrc1 = two ? M.wavelet[n + 1] * M.vol_inv : 0.f;

    // ---- incident, first level on E
    for (int g = tid; g < kTbGroups; g += kThreads) {
        const int er = g / (kTbEX / 4), ec = (g - er * (kTbEX / 4)) * 4;
        const int z = z0 - 4 + er, x = x0 - 4 + ec;
        float L[4], o[4], d[4];
        float4 c;
        lap4<kTbHX>(U0, er + 4, ec + 4, M, c, L);
        tb_incident4(M, c, L, ld4(S + er * kTbEX + ec), ld4(U1 + er * kTbEX + ec), z, x, z >= 0 && z < M.Nz, sz, sx,
                     fsrc0, o, d);
        st4(UN + er * kTbEX + ec, make_float4(o[0], o[1], o[2], o[3]));
        st4(DN + er * kTbEX + ec, make_float4(d[0], d[1], d[2], d[3]));
    }
    __syncthreads();

    // ---- incident, second level on the tile
    const int lx = (tid & 15) << 2, lz = tid >> 4;
    const int z = z0 + lz, x = x0 + lx;
    const bool valid = (z < M.Nz) && (x < M.Nx);
    const long long off = (long long)z * M.P + x;
    const int te = (lz + 4) * kTbEX + lx + 4;  // this thread's cells in the E arrays
    const int th = (lz + 8) * kTbHX + lx + 8;  // and in the tile + 8 arrays
    const float4 sv = ld4(S + te);
    float d1[4] = {0.f, 0.f, 0.f, 0.f};
    float* u4 = M.u4 + (long long)(shot * 4) * F;
    if (two) {
        float L[4], o[4];
        float4 c1;
        lap4<kTbEX>(UN, lz + 4, lx + 4, M, c1, L);
        tb_incident4(M, c1, L, sv, ld4(U0 + th), z, x, true, sz, sx, fsrc1, o, d1);
        if (valid) {
            st4(u4 + p1 * F + off, c1);
            st4(u4 + p2 * F + off, make_float4(o[0], o[1], o[2], o[3]));
        }
    } else if (valid) {
        st4(u4 + p1 * F + off, ld4(UN + te));
    }
    if ((DTT || (BORN && M.dtt_store)) && valid) {
        float* dst = M.dtt + (long long)shot * M.dtt_shot_stride + off;
        st4(dst + (long long)M.dtt_slot * F, ld4(DN + te));
        if (two) st4(dst + (long long)(M.dtt_slot + 1) * F, make_float4(d1[0], d1[1], d1[2], d1[3]));
    }
    if (!BORN) return;

    const int nb = M.nb;
    for (int b = 0; b < nb; ++b) {
        __syncthreads();  // the previous trial is done with F0, F1, DM, FN
        if (tid == 0) {
            mbar_expect_tx(&bars[1], kTbLoadBytes);
            tma_load_3d(F0, &M.tm_f4h, x0 - 8, z0 - 8, (shot * nb + b) * 4 + pn, &bars[1]);
            tma_load_3d(F1, &M.tm_f4e, x0 - 4, z0 - 4, (shot * nb + b) * 4 + pm, &bars[1]);
            tma_load_3d(DM, &M.tm_dme, x0 - 4, z0 - 4, b, &bars[1]);
        }
        const bool ok = mbar_wait_bounded(&bars[1], (uint32_t)(b & 1));
        if (__syncthreads_or(!ok)) {
            const uint32_t par[1] = {(uint32_t)(b & 1)};
            abort_cta(p.err, bars + 1, 1, par);
            return;
        }
        float* dout = M.data + (long long)shot * M.data_shot_stride + (long long)b * M.data_trial_stride;
        tb_sample<kTbHX>(F0, 8, M, tile, z0, x0, dout + (long long)n * M.nr);
        for (int g = tid; g < kTbGroups; g += kThreads) {
            const int er = g / (kTbEX / 4), ec = (g - er * (kTbEX / 4)) * 4;
            const int zz = z0 - 4 + er, xx = x0 - 4 + ec;
            float L[4], o[4];
            float4 c;
            lap4<kTbHX>(F0, er + 4, ec + 4, M, c, L);
            const float4 dd = ld4(DN + er * kTbEX + ec);
            const float dv4[4] = {dd.x, dd.y, dd.z, dd.w};
            tb_born4(M, c, L, ld4(S + er * kTbEX + ec), ld4(F1 + er * kTbEX + ec), ld4(DM + er * kTbEX + ec), dv4,
                     zz, xx, zz >= 0 && zz < M.Nz, o);
            st4(FN + er * kTbEX + ec, make_float4(o[0], o[1], o[2], o[3]));
        }
        __syncthreads();
        float* f4 = M.f4 + (long long)((shot * nb + b) * 4) * F;
        if (two) {
            tb_sample<kTbEX>(FN, 4, M, tile, z0, x0, dout + (long long)(n + 1) * M.nr);
            float L[4], o[4];
            float4 c1;
            lap4<kTbEX>(FN, lz + 4, lx + 4, M, c1, L);
            tb_born4(M, c1, L, sv, ld4(F0 + th), ld4(DM + te), d1, z, x, true, o);
            if (valid) {
                st4(f4 + p1 * F + off, c1);
                st4(f4 + p2 * F + off, make_float4(o[0], o[1], o[2], o[3]));
            }
        } else if (valid) {
            st4(f4 + p1 * F + off, ld4(FN + te));
        }
    }
}

cudaError_t launch_fwd2d_tb(FwdKind kind, const StepParams2D& p, int zblocks, cudaStream_t st) {
    if (zblocks <= 0) return cudaSuccess;
    const dim3 grid = grid2d(p, zblocks);
    const size_t sm = fwd2d_tb_smem_bytes();
    cudaError_t e;
    switch (kind) {
        case FWD_BORN:
            e = cudaFuncSetAttribute(k_fwd2d_tb<FWD_BORN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            k_fwd2d_tb<FWD_BORN><<<grid, kThreads, sm, st>>>(p);
            break;
        case FWD_INCIDENT_DTT:
            e = cudaFuncSetAttribute(k_fwd2d_tb<FWD_INCIDENT_DTT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            k_fwd2d_tb<FWD_INCIDENT_DTT><<<grid, kThreads, sm, st>>>(p);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t stencil2d_configure() { return cudaSuccess; }

}  // namespace probe
