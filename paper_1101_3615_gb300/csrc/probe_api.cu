// C ABI of the matrix-probing library: handle life cycle, argument validation,
// memory planning, TMA descriptors, and the orchestration of the sweeps that
// make up F, F*, H = F*F (Sec. 1.1, Sec. 2), the nonlinear forward map and the
// misfit gradient.  Every arithmetic step runs in the sm_103a kernels of
// stencil2d.cu / aux.cu / fit.cu; this file only launches them.
//
// Sweep structure of one wave of resident shots (all on one stream):
//   forward   n = 0..nt-2: one fused launch per step (incident field u0 and nb
//             Born fields), checkpoint (u^n, u^{n-1}) every K steps, receivers
//             sampled in-kernel; the last level sampled by a small kernel.
//   adjoint   checkpoint segments in reverse: restore (u^{k0}, u^{k0-1}),
//             recompute u^{k0..k1-1} writing Dtt u^n into the segment buffer,
//             then run the adjoint recurrence n = k1..k0+1 with receiver
//             injection and the fused imaging condition.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "internal.h"

using namespace probe;

namespace {

thread_local std::string g_create_error;

}  // namespace

namespace probe {

probe_status fail(probe_t h, probe_status st, const std::string& msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return st;
}

probe_status cuda_fail(probe_t h, cudaError_t e, const char* what) {
    const probe_status st = (e == cudaErrorMemoryAllocation) ? PROBE_ERR_OOM : PROBE_ERR_CUDA;
    return fail(h, st, std::string(what) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

probe_status ensure_buf(probe_t h, DevBuf& b, size_t bytes) {
    if (b.n >= bytes) return PROBE_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    PROBE_CK(h, cudaMalloc(&b.p, bytes));
    b.n = bytes;
    return PROBE_OK;
}

}  // namespace probe

#define CK(h, call) PROBE_CK(h, call)
#define TRY(call) PROBE_TRY(call)

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

probe_status get_encoder(probe_t h) {
    if (g_encode) return PROBE_OK;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    CK(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn)
        return fail(h, PROBE_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return PROBE_OK;
}

// 3D FP32 tensor map over `planes` planes of [Nz][P] floats (extent Nx in x) with a
// (64 + 8) x (tile_z + 8) box; out-of-range elements read as zero.
probe_status encode_planes(probe_t h, CUtensorMap* map, float* base, int planes, int tile_z) {
    TRY(get_encoder(h));
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r;
    if (h->ndim == 2) {
        cuuint64_t dims[3] = {(cuuint64_t)h->Nx, (cuuint64_t)h->Nz, (cuuint64_t)planes};
        cuuint64_t strides[2] = {(cuuint64_t)h->P * 4, (cuuint64_t)h->F * 4};
        cuuint32_t box[3] = {(cuuint32_t)(kTX + 8), (cuuint32_t)(tile_z + 8), 1};
        r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        // (x, y, z, volume) with a one-plane (64 + 8) x (16 + 8) box
        cuuint64_t dims[4] = {(cuuint64_t)h->Nx, (cuuint64_t)h->Ny, (cuuint64_t)h->Nz, (cuuint64_t)planes};
        cuuint64_t strides[3] = {(cuuint64_t)h->P * 4, (cuuint64_t)h->Ny * h->P * 4, (cuuint64_t)h->F * 4};
        cuuint32_t box[4] = {(cuuint32_t)(kTX + 8), (cuuint32_t)(kTY3D + 8), 1, 1};
        r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS)
        return fail(h, PROBE_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return PROBE_OK;
}

// 2D FP32 tensor map over `planes` planes with a bx x bz box (the time-blocked kernels' boxes).
probe_status encode_box(probe_t h, CUtensorMap* map, const float* base, int planes, int bx, int bz) {
    TRY(get_encoder(h));
    cuuint32_t es[3] = {1, 1, 1};
    cuuint64_t dims[3] = {(cuuint64_t)h->Nx, (cuuint64_t)h->Nz, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)h->P * 4, (cuuint64_t)h->F * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)bz, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(h, PROBE_ERR_CUDA, "cuTensorMapEncodeTiled (box) failed (" + std::to_string((int)r) + ")");
    return PROBE_OK;
}

// 2D FP32 tensor map over `planes` planes with a plain 64 x rows box (no halo).
probe_status encode_plain(probe_t h, CUtensorMap* map, const float* base, int planes, int rows) {
    TRY(get_encoder(h));
    cuuint32_t es[3] = {1, 1, 1};
    cuuint64_t dims[3] = {(cuuint64_t)h->Nx, (cuuint64_t)h->Nz, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)h->P * 4, (cuuint64_t)h->F * 4};
    cuuint32_t box[3] = {(cuuint32_t)kTX, (cuuint32_t)rows, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(h, PROBE_ERR_CUDA, "cuTensorMapEncodeTiled (plain box) failed (" + std::to_string((int)r) + ")");
    return PROBE_OK;
}

// Workspace generations are unique in the process, so a cached graph keyed by
// (handle, generation) can never match a later workspace at reused addresses.
std::atomic<long long> g_generation{0};

void free_ws(Workspace& w) {
    void* ptrs[] = {w.u, w.f, w.dm, w.data, w.ckpt, w.scales, w.absmax, w.dtt, w.img, w.comp, w.s_tmp,
                    w.src_wave, w.inj, w.seg, w.u4, w.f4};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    w = Workspace();
    w.generation = ++g_generation;
}


// Floats of one (slot, shot, trial) block of the adjoint injection buffer: the grid rows (2D) or
// planes (3D) that hold receivers.
long long inj_block(probe_t h) { return (long long)h->nband * (h->ndim == 3 ? (long long)h->Ny * h->P : h->P); }

// Bytes per resident shot and fixed bytes of a job with nb trials.
bool use_history(probe_t h, int with_ckpt) { return with_ckpt && h->opt_dtt_history && h->ndim == 2; }

// 3D adjoint on the producer-warp kernel (receiver injection from a per-segment band buffer)
// rather than the one-barrier-per-plane kernel or the shot-cluster kernel.
bool adj3d_ws(probe_t h) { return h->ndim == 3 && h->pipe_adj != 0 && !(h->opt_cluster3d & 2); }

void ws_bytes(probe_t h, int nb, int with_ckpt, int with_data, double* per_shot, double* fixed) {
    const double F4 = (double)h->F * 4.0;
    double ps = 2 * F4 + 2.0 * nb * F4;
    if (h->ndim == 2) ps += 4 * F4 + 4.0 * nb * F4;  // four-level states of the time-blocked forward
    if (use_history(h, with_ckpt))
        ps += (double)(h->nt - 1) * F4;
    else if (with_ckpt)
        ps += (double)h->nck * ckpt_bytes_per_shot(h->snap, h->F) + (double)h->K * F4 + 16.0 * h->nck;
    else if (h->ndim == 3)
        ps += 2.0 * F4;  // Dtt u^n of two steps (Born source)
    if (with_data) ps += (double)nb * h->nt * h->nr * 4.0;
    if (h->ndim == 3 && with_ckpt) {
        ps += 2.0 * nb * F4;  // per-shot images + compensation
        if ((h->opt_cluster3d & 2) || adj3d_ws(h)) ps += (double)h->K * nb * inj_block(h) * 4.0;  // injection of one segment
        if (!(h->opt_cluster3d & 2) && h->kahan) ps += (double)nb * F4;                          // segment images
    }
    *per_shot = ps;
    *fixed = nb * F4 + 2.0 * F4 * nb + F4;  // dm, one image group, s_tmp
}

int plan_wave(probe_t h, int nb, int with_ckpt, int with_data) {
    if (h->opt_shot_wave > 0) return std::min(h->opt_shot_wave, h->ns);
    double ps, fx;
    ws_bytes(h, nb, with_ckpt, with_data, &ps, &fx);
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    const double budget = 0.80 * (double)freeb + (double)h->ws.bytes;
    int W = std::max(1, std::min((int)std::floor((budget - fx) / ps), h->ns));
    // equal waves: the fewest waves that fit, with the shots spread evenly over them (so that the
    // last wave is not a remainder of one or two shots)
    const int nwaves = (h->ns + W - 1) / W;
    return (h->ns + nwaves - 1) / nwaves;
}

int pick_group(probe_t h, int W) {
    if (h->ndim == 3) {
        // one-field kernels: one image per shot and trial; cluster kernels: clusters of g shots,
        // g in {1, 2, 4, 8} dividing every wave (the full waves and the last one)
        if (!(h->opt_cluster3d & 2)) return 1;
        const int last = (h->ns % W) ? h->ns % W : W;
        int g = h->opt_shot_group > 0 ? std::min(h->opt_shot_group, 8) : 4;
        while (g > 1 && ((g & (g - 1)) || W % g || last % g)) --g;
        return std::max(g, 1);
    }
    if (h->opt_shot_group > 0) return std::min(h->opt_shot_group, W);
    return std::min(4, W);
}

// Tensor maps of the pipelined kernels for tiles of 64 x 16R (host-side encoding only).
probe_status encode_ws_maps(probe_t h, WsMaps& m, int R) {
    Workspace& w = h->ws;
    const int rows = 16 * R;
    const int nb = std::max(w.nb, 1);
    TRY(encode_planes(h, &m.wu, w.u, w.W * 2, rows));
    TRY(encode_planes(h, &m.wf, w.f, w.W * nb * 2, rows));
    TRY(encode_plain(h, &m.up, w.u, w.W * 2, rows));
    TRY(encode_plain(h, &m.fp, w.f, w.W * nb * 2, rows));
    TRY(encode_plain(h, &m.dmp, w.dm, nb, rows));
    if (w.dtt) TRY(encode_plain(h, &m.dtp, w.dtt, w.W * w.dtt_slots, rows));
    if (w.img) {
        TRY(encode_plain(h, &m.img, w.img, w.groups * nb, rows));
        TRY(encode_plain(h, &m.cmp, w.comp, w.groups * nb, rows));
    }
    m.rows = R;
    return PROBE_OK;
}

probe_status ensure_ws(probe_t h, int W, int nb, int with_ckpt, int with_data) {
    Workspace& w = h->ws;
    const int G = W;  // image groups for the smallest shot group: any group size fits
    const int history = use_history(h, with_ckpt) ? 1 : 0;
    if (w.u && w.W >= W && w.nb >= nb && w.with_ckpt >= with_ckpt && w.with_data >= with_data &&
        w.groups >= G && w.tm_tile_z == h->tile_z && w.W == W && w.nb == nb && w.history == history)
        return PROBE_OK;
    free_ws(w);
    const long long F = h->F;
    auto alloc = [&](void** p, size_t bytes) -> probe_status {
        if (bytes == 0) return PROBE_OK;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            free_ws(w);
            return cuda_fail(h, e, "workspace allocation");
        }
        w.bytes += bytes;
        return PROBE_OK;
    };
    TRY(alloc((void**)&w.u, (size_t)W * 2 * F * 4));
    TRY(alloc((void**)&w.f, (size_t)W * std::max(nb, 1) * 2 * F * 4));
    TRY(alloc((void**)&w.dm, (size_t)std::max(nb, 1) * F * 4));
    if (with_data) TRY(alloc((void**)&w.data, (size_t)W * nb * h->nt * h->nr * 4));
    if (history) {
        TRY(alloc((void**)&w.dtt, (size_t)W * (h->nt - 1) * F * 4));  // Dtt u^n of every step
    } else if (with_ckpt) {
        TRY(alloc(&w.ckpt, (size_t)h->nck * W * ckpt_bytes_per_shot(h->snap, F)));
        TRY(alloc((void**)&w.scales, (size_t)h->nck * W * 2 * 4));
        TRY(alloc((void**)&w.absmax, (size_t)W * 2 * 4));
        TRY(alloc((void**)&w.dtt, (size_t)W * h->K * F * 4));
    } else if (h->ndim == 3) {
        TRY(alloc((void**)&w.dtt, (size_t)W * 2 * F * 4));  // Dtt u^n of two steps (Born source)
    }
    TRY(alloc((void**)&w.img, (size_t)G * std::max(nb, 1) * F * 4));
    TRY(alloc((void**)&w.comp, (size_t)G * std::max(nb, 1) * F * 4));
    if (h->ndim == 3 && with_ckpt && h->kahan && !(h->opt_cluster3d & 2)) {
        TRY(alloc((void**)&w.seg, (size_t)W * std::max(nb, 1) * F * 4));
        CK(h, cudaMemset(w.seg, 0, (size_t)W * std::max(nb, 1) * F * 4));  // pitch columns stay zero
    }
    TRY(alloc((void**)&w.s_tmp, (size_t)F * 4));
    TRY(alloc((void**)&w.src_wave, (size_t)W * 3 * 4));
    if (with_ckpt && h->nband > 0 && (h->ndim == 2 || (h->opt_cluster3d & 2) || adj3d_ws(h)))  // one segment of adjoint injection
        TRY(alloc((void**)&w.inj, (size_t)h->K * W * std::max(nb, 1) * inj_block(h) * 4));
    // field planes must read as zero outside what the kernels write
    CK(h, cudaMemset(w.u, 0, (size_t)W * 2 * F * 4));
    CK(h, cudaMemset(w.f, 0, (size_t)W * std::max(nb, 1) * 2 * F * 4));
    w.history = history;
    w.dtt_slots = history ? h->nt - 1 : (with_ckpt ? h->K : (h->ndim == 3 ? 2 : 1));
    if (w.dtt) CK(h, cudaMemset(w.dtt, 0, (size_t)W * w.dtt_slots * F * 4));
    w.W = W;
    w.nb = nb;
    w.with_ckpt = with_ckpt;
    w.with_data = with_data;
    w.groups = G;
    TRY(encode_planes(h, &w.tm_u, w.u, W * 2, h->tile_z));
    TRY(encode_planes(h, &w.tm_f, w.f, W * std::max(nb, 1) * 2, h->tile_z));
    if (h->ndim == 2) {
        TRY(encode_ws_maps(h, w.mf, h->ws_rows));
        TRY(encode_ws_maps(h, w.ma, h->ws_rows_adj));
        // four-level states of the time-blocked forward (zero: levels -1 and 0 start at rest)
        TRY(alloc((void**)&w.u4, (size_t)W * 4 * F * 4));
        TRY(alloc((void**)&w.f4, (size_t)W * std::max(nb, 1) * 4 * F * 4));
        CK(h, cudaMemset(w.u4, 0, (size_t)W * 4 * F * 4));
        CK(h, cudaMemset(w.f4, 0, (size_t)W * std::max(nb, 1) * 4 * F * 4));
        TRY(encode_box(h, &w.tm_u4h, w.u4, W * 4, kTX + 16, 32));
        TRY(encode_box(h, &w.tm_u4e, w.u4, W * 4, kTX + 8, 24));
        TRY(encode_box(h, &w.tm_f4h, w.f4, W * std::max(nb, 1) * 4, kTX + 16, 32));
        TRY(encode_box(h, &w.tm_f4e, w.f4, W * std::max(nb, 1) * 4, kTX + 8, 24));
        TRY(encode_box(h, &w.tm_dme, w.dm, std::max(nb, 1), kTX + 8, 24));
    }
    w.tm_tile_z = h->tile_z;
    return PROBE_OK;
}

// Receivers bucketed by key (CSR: ptr [nkeys + 1], idx [nr]) uploaded to *ptr / *idx.
probe_status upload_csr(probe_t h, const std::vector<int>& key, int nkeys, int** ptr, int** idx_out) {
    std::vector<int> cnt(nkeys + 1, 0), idx(h->nr);
    for (int r = 0; r < h->nr; ++r) cnt[key[r] + 1]++;
    for (int t = 0; t < nkeys; ++t) cnt[t + 1] += cnt[t];
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int r = 0; r < h->nr; ++r) idx[pos[key[r]]++] = r;
    if (*ptr) cudaFree(*ptr);
    if (*idx_out) cudaFree(*idx_out);
    *ptr = *idx_out = nullptr;
    CK(h, cudaMalloc(ptr, cnt.size() * 4));
    CK(h, cudaMalloc(idx_out, std::max<size_t>(idx.size(), 1) * 4));
    CK(h, cudaMemcpy(*ptr, cnt.data(), cnt.size() * 4, cudaMemcpyHostToDevice));
    if (!idx.empty()) CK(h, cudaMemcpy(*idx_out, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice));
    return PROBE_OK;
}

// 2D adjoint injection layout: the grid rows that hold receivers (bands) and the distinct
// receiver cells with their receivers in receiver order (so sums are formed in a fixed order).
// 3D: the same with the z planes that hold receivers as bands, position band * Ny * P + y * P + x.
probe_status build_bands(probe_t h) {
    const int d = h->ndim;
    std::vector<int> rrow(h->Nz, -1);
    int nband = 0;
    for (int r = 0; r < h->nr; ++r) {
        const int z = h->rec_pad[d * r];
        if (rrow[z] < 0) rrow[z] = 0;
    }
    for (int z = 0; z < h->Nz; ++z)
        if (rrow[z] == 0) rrow[z] = nband++;
    const long long plane = (d == 3) ? (long long)h->Ny * h->P : h->P;
    std::map<std::pair<int, long long>, std::vector<int>> cells;  // (band, cell in the band) -> receivers
    for (int r = 0; r < h->nr; ++r) {
        const long long in_band = (d == 3) ? (long long)h->rec_pad[3 * r + 1] * h->P + h->rec_pad[3 * r + 2]
                                           : h->rec_pad[2 * r + 1];
        cells[{rrow[h->rec_pad[d * r]], in_band}].push_back(r);
    }
    std::vector<int> ptr(1, 0), rec, pos;
    for (const auto& kv : cells) {
        for (int r : kv.second) rec.push_back(r);
        ptr.push_back((int)rec.size());
        pos.push_back((int)(kv.first.first * plane + kv.first.second));
    }
    auto upload = [&](int** dst, const std::vector<int>& v) -> probe_status {
        CK(h, cudaMalloc(dst, std::max<size_t>(v.size(), 1) * 4));
        if (!v.empty()) CK(h, cudaMemcpy(*dst, v.data(), v.size() * 4, cudaMemcpyHostToDevice));
        return PROBE_OK;
    };
    TRY(upload(&h->d_rrow, rrow));
    TRY(upload(&h->d_uc_ptr, ptr));
    TRY(upload(&h->d_uc_rec, rec));
    TRY(upload(&h->d_uc_pos, pos));
    h->nband = nband;
    h->nuc = (int)pos.size();
    return PROBE_OK;
}

// Receivers grouped by 2D tile (CSR) for the in-tile sampling and injection.
probe_status build_rec_tiles(probe_t h) {
    std::vector<int> key(h->nr);
    int nkeys;
    if (h->ndim == 2) {
        h->tiles_x = (h->Nx + kTX - 1) / kTX;
        h->tiles_z = (h->Nz + h->tile_z - 1) / h->tile_z;
        h->ntiles = h->tiles_x * h->tiles_z;
        nkeys = h->ntiles;
        for (int r = 0; r < h->nr; ++r) {
            const int z = h->rec_pad[2 * r], x = h->rec_pad[2 * r + 1];
            key[r] = (z / h->tile_z) * h->tiles_x + x / kTX;
        }
    } else {
        h->tiles_x = (h->Nx + kTX - 1) / kTX;
        h->tiles_y = (h->Ny + kTY3D - 1) / kTY3D;
        h->tiles_z = (h->Nz + kZC3D - 1) / kZC3D;
        h->ntiles = h->tiles_x * h->tiles_y * h->tiles_z;
        nkeys = h->tiles_x * h->tiles_y * h->Nz;
        for (int r = 0; r < h->nr; ++r) {
            const int z = h->rec_pad[3 * r], y = h->rec_pad[3 * r + 1], x = h->rec_pad[3 * r + 2];
            key[r] = ((y / kTY3D) * h->tiles_x + x / kTX) * h->Nz + z;
        }
    }
    TRY(upload_csr(h, key, nkeys, &h->d_rec_tile_ptr, &h->d_rec_tile_idx));
    if (!h->d_rrow) TRY(build_bands(h));
    if (h->ndim == 2) {
        for (int R = 1; R <= 2; ++R) {  // tiles of the pipelined kernels (64 x 16R)
            const int tz = (h->Nz + 16 * R - 1) / (16 * R);
            for (int r = 0; r < h->nr; ++r)
                key[r] = (h->rec_pad[2 * r] / (16 * R)) * h->tiles_x + h->rec_pad[2 * r + 1] / kTX;
            TRY(upload_csr(h, key, tz * h->tiles_x, &h->d_wrec_ptr[R], &h->d_wrec_idx[R]));
        }
    }
    return PROBE_OK;
}

probe_status set_tile_z(probe_t h, int tz) {
    if (tz == h->tile_z && h->d_rec_tile_ptr) return PROBE_OK;
    h->tile_z = tz;
    TRY(build_rec_tiles(h));
    free_ws(h->ws);  // tensor-map boxes depend on the tile height
    return PROBE_OK;
}

// ---------------------------------------------------------------------------
// Sweeps over a list of jobs (one per model) that advance in the same launches.
// ---------------------------------------------------------------------------
struct Job {
    probe_t h;
    int j0 = 0, W = 0, nb = 0;
    const float* s = nullptr;
    float* data = nullptr;          // forward output (Born or incident traces), may be null
    const float* rdata = nullptr;   // adjoint input
    long long dss = 0, dts = 0;     // data strides: shot, trial
    int groups = 1, shot_group = 1;
};

// One model's parameter block; maps: the pipelined-kernel tensor maps (forward or adjoint set).
void fill_model(const Job& jb, ModelStep2D& m, const WsMaps& maps, int* blocks_fwd, int* blocks_adj) {
    probe_t h = jb.h;
    Workspace& w = h->ws;
    m.tm_u = w.tm_u;
    m.tm_f = w.tm_f;
    m.tm_wu = maps.wu;
    m.tm_wf = maps.wf;
    m.tm_up = maps.up;
    m.tm_fp = maps.fp;
    m.tm_dmp = maps.dmp;
    m.tm_dtp = maps.dtp;
    m.tm_img = maps.img;
    m.tm_cmp = maps.cmp;
    m.dtt_slots = w.dtt_slots;
    m.dtt_store = w.history;
    const int R = maps.rows > 0 ? maps.rows : 1;
    m.ws_rows = R;
    m.ws_tiles_z = (h->Nz + 16 * R - 1) / (16 * R);
    m.ws_ntiles = m.ws_tiles_z * h->tiles_x;
    m.ws_rec_ptr = h->d_wrec_ptr[R];
    m.ws_rec_idx = h->d_wrec_idx[R];
    m.rrow = h->d_rrow;
    m.inj = w.inj;
    m.nband = h->nband;
    m.inj_slot = 0;
    if (encode_plain(h, &m.tm_sp, jb.s, 1, 16 * R) != PROBE_OK) m.s = nullptr;
    m.tm_u4h = w.tm_u4h;
    m.tm_u4e = w.tm_u4e;
    m.tm_f4h = w.tm_f4h;
    m.tm_f4e = w.tm_f4e;
    m.tm_dme = w.tm_dme;
    if (w.u4 && encode_box(h, &m.tm_se, jb.s, 1, kTX + 8, 24) != PROBE_OK) m.s = nullptr;
    m.u4 = w.u4;
    m.f4 = w.f4;
    m.Nz = h->Nz;
    m.Nx = h->Nx;
    m.P = h->P;
    m.pad = h->pad;
    m.nz = h->nz;
    m.nx = h->nx;
    m.tiles_x = h->tiles_x;
    m.tiles_z = h->tiles_z;
    m.ntiles = h->ntiles;
    m.nshots = jb.W;
    m.nb = jb.nb;
    m.shot_group = jb.shot_group;
    m.ngroups = jb.groups;
    m.nbc_chunks = 1;
    m.nr = h->nr;
    m.dtt_slot = 0;
    m.cz = h->cz;
    m.cx = h->cx;
    const double w0 = PROBE_W0, wk[4] = {PROBE_W1, PROBE_W2, PROBE_W3, PROBE_W4};
    m.c0 = (float)(w0 / (h->hz * h->hz) + w0 / (h->hx * h->hx));
    for (int k = 0; k < 4; ++k) {
        m.lz[k] = (float)(wk[k] / (h->hz * h->hz));
        m.lx[k] = (float)(wk[k] / (h->hx * h->hx));
    }
    for (int mm = 0; mm < 4; ++mm) {
        double cm = 0.0;
        for (int k = mm; k < 4; ++k) cm += wk[k];
        m.cxm[mm] = (float)(cm / (h->hx * h->hx));
        m.czm[mm] = (float)(cm / (h->hz * h->hz));
    }
    m.inv_dt2 = (float)(1.0 / (h->dt * h->dt));
    m.vol_inv = (float)(1.0 / (h->hz * h->hx));
    m.F = h->F;
    m.u = w.u;
    m.f = w.f;
    m.s = jb.s;
    m.dm = w.dm;
    m.dtt = w.dtt;
    m.dtt_shot_stride = (long long)w.dtt_slots * h->F;
    m.wavelet = h->d_wavelet;
    m.src_zx = w.src_wave;
    m.rec_tile_ptr = h->d_rec_tile_ptr;
    m.rec_tile_idx = h->d_rec_tile_idx;
    m.rec_zx = h->d_rec;
    m.data = jb.data;
    m.rdata = jb.rdata;
    m.data_shot_stride = jb.dss;
    m.data_trial_stride = jb.dts;
    m.img = w.img;
    m.comp = w.comp;
    m.img_group_stride = (long long)std::max(w.nb, 1) * h->F;
    *blocks_fwd = jb.W;        // grid.z extent of the forward launches
    *blocks_adj = jb.groups;   // grid.z extent of the adjoint launches
}

struct Sweep {
    std::vector<Job> jobs;
    StepParams2D p;   // forward launches
    StepParams2D pa;  // adjoint launches (the pipelined adjoint may use another tile height)
    int blocks_fwd = 0, blocks_adj = 0;
    int nbc = 1, chunks = 1;
    int tile_z = 16;
    int pipeline = 0;      // forward: 0 one tile per CTA; 2..4 persistent pipelined kernels
    int pipeline_adj = 0;  // adjoint variant
    int inj_hi = -1;       // time level of injection slot 0 of the current segment (-1: slot 0)
    int tb = 1;            // Born forward and recompute: time levels per launch (1 or 2)
    bool kahan = true;
    cudaStream_t st = nullptr;
    int nt = 0, K = 0, nck = 0;
    long long launches_fwd = 0, launches_rec = 0, launches_adj = 0, launches_other = 0;
};

probe_status prepare_sweep(Sweep& sw, probe_t h0, cudaStream_t st) {
    memset(&sw.p, 0, sizeof(sw.p));
    sw.p.nmodels = (int)sw.jobs.size();
    sw.p.nt = h0->nt;
    sw.p.err = h0->d_err;
    memset(&sw.pa, 0, sizeof(sw.pa));
    sw.pa.nmodels = sw.p.nmodels;
    sw.pa.nt = sw.p.nt;
    sw.pa.err = sw.p.err;
    sw.st = st;
    sw.nt = h0->nt;
    sw.K = h0->K;
    sw.nck = h0->nck;
    sw.tile_z = h0->tile_z;
    sw.pipeline = h0->opt_pipeline;
    sw.pipeline_adj = h0->pipe_adj;
    sw.tb = (h0->ndim == 2 && h0->tile_z == kPipeTZ && h0->ws.u4) ? h0->opt_tblock : 1;
    sw.kahan = h0->kahan != 0;
    int maxnb = 1;
    std::vector<int> bf(sw.jobs.size()), ba(sw.jobs.size());
    for (Job& jb : sw.jobs) {  // every model of a launch uses the first one's pipelined tile heights
        Workspace& w = jb.h->ws;
        if (jb.h->ndim != 2 || !w.u) continue;
        if (w.mf.rows != h0->ws_rows) TRY(encode_ws_maps(jb.h, w.mf, h0->ws_rows));
        if (w.ma.rows != h0->ws_rows_adj) TRY(encode_ws_maps(jb.h, w.ma, h0->ws_rows_adj));
    }
    for (size_t k = 0; k < sw.jobs.size(); ++k) {
        int f, a;
        fill_model(sw.jobs[k], sw.pa.m[k], sw.jobs[k].h->ws.ma, &f, &a);
        fill_model(sw.jobs[k], sw.p.m[k], sw.jobs[k].h->ws.mf, &f, &a);
        bf[k] = f;
        ba[k] = a;
        maxnb = std::max(maxnb, sw.jobs[k].nb);
    }
    sw.nbc = maxnb <= 1 ? 1 : (maxnb <= 2 ? 2 : (maxnb <= 4 ? 4 : 8));
    if (sw.pipeline_adj && sw.tile_z == kPipeTZ && h0->ws_rows_adj == 2) sw.nbc = std::min(sw.nbc, 4);
    sw.chunks = (maxnb + sw.nbc - 1) / sw.nbc;
    // block_begin differs between the forward and the adjoint grids; kept for
    // the forward here and rewritten by set_grid().
    sw.blocks_fwd = 0;
    sw.blocks_adj = 0;
    for (size_t k = 0; k < sw.jobs.size(); ++k) {
        sw.blocks_fwd += bf[k];
        sw.blocks_adj += ba[k];
    }
    return PROBE_OK;
}

void set_grid(Sweep& sw, bool adjoint) {
    const bool ws = (adjoint ? sw.pipeline_adj : sw.pipeline) && sw.tile_z == kPipeTZ;
    StepParams2D& p = adjoint ? sw.pa : sw.p;
    int b = 0, items = 0;
    for (size_t k = 0; k < sw.jobs.size(); ++k) {
        const Job& jb = sw.jobs[k];
        const int units = adjoint ? jb.groups : jb.W;
        p.m[k].block_begin = b;
        p.m[k].item_begin = items;
        b += units;
        items += units * (ws ? p.m[k].ws_ntiles : jb.h->ntiles);
    }
    p.total_items = items;
}

probe_status launch_fwd_step(Sweep& sw, FwdKind kind, int n, int slot) {
    set_grid(sw, false);
    sw.p.n = n;
    for (int k = 0; k < sw.p.nmodels; ++k) sw.p.m[k].dtt_slot = slot;
    cudaError_t e = (sw.pipeline && sw.tile_z == kPipeTZ) ? launch_fwd2d_pipe(kind, sw.pipeline, sw.p, sw.st)
                                                           : launch_fwd2d(kind, sw.tile_z, sw.p, sw.blocks_fwd, sw.st);
    if (e != cudaSuccess) return cuda_fail(sw.jobs[0].h, e, "forward step launch");
    return PROBE_OK;
}

// Kernel launches of one checkpoint store (encode) or restore: FP32 copies are a plain memory copy
// when the state planes are already in checkpoint order (u^n first).
int codec_launches(int snap, bool encode, int pps, int p_un) {
    if (snap == PROBE_SNAP_FP32) return (pps == 2 && p_un == 0) ? 0 : 1;
    return encode ? 2 : 1;
}

// Time-blocked forward launch: levels n -> n + 2 (two) or n -> n + 1, Dtt into slots slot, slot + 1.
probe_status launch_fwd_tb(Sweep& sw, FwdKind kind, int n, bool two, int slot) {
    set_grid(sw, false);
    sw.p.n = n;
    sw.p.two = two ? 1 : 0;
    for (int k = 0; k < sw.p.nmodels; ++k) sw.p.m[k].dtt_slot = slot;
    cudaError_t e = launch_fwd2d_tb(kind, sw.p, sw.blocks_fwd, sw.st);
    if (e != cudaSuccess) return cuda_fail(sw.jobs[0].h, e, "time-blocked forward launch");
    return PROBE_OK;
}

probe_status launch_adj_step(Sweep& sw, int n, int slot) {
    set_grid(sw, true);
    sw.pa.n = n;
    for (int k = 0; k < sw.pa.nmodels; ++k) {
        sw.pa.m[k].dtt_slot = slot;
        sw.pa.m[k].inj_slot = sw.inj_hi >= 0 ? sw.inj_hi - n : 0;
    }
    cudaError_t e = (sw.pipeline_adj && sw.tile_z == kPipeTZ)
                        ? launch_adj2d_pipe(sw.nbc, sw.kahan, sw.pipeline_adj, sw.pa, sw.chunks, sw.st)
                        : launch_adj2d(sw.tile_z, sw.nbc, sw.kahan, sw.pa, sw.blocks_adj, sw.chunks, sw.st);
    if (e != cudaSuccess) return cuda_fail(sw.jobs[0].h, e, "adjoint step launch");
    return PROBE_OK;
}

void record(probe_t h, int idx, cudaStream_t st) {
    // external: inside a stream capture the record becomes an event node of the graph
    if (!h->opt_timing || (h->opt_timing == 2 && idx > 1)) return;  // level 2: the forward sweep only
    idx += h->ev_base;
    if (idx >= (int)h->events.size()) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(h->events[idx], st, cudaEventRecordExternal);
    else
        cudaEventRecord(h->events[idx], st);
}

// Forward sweep.  kind: FWD_BORN / FWD_INCIDENT / FWD_INCIDENT_SAMPLE.
// Born forward with two time levels per launch over the four-level states (levels n, n - 1 read,
// n + 1, n + 2 written); checkpoints are taken between launches, where (u^m, u^{m-1}) of every m
// the launch reached are in the planes m & 3, (m - 1) & 3.
probe_status run_forward_tb(Sweep& sw, bool ckpt) {
    for (Job& jb : sw.jobs) {
        Workspace& w = jb.h->ws;
        CK(jb.h, cudaMemsetAsync(w.u4, 0, (size_t)jb.W * 4 * jb.h->F * 4, sw.st));
        CK(jb.h, cudaMemsetAsync(w.f4, 0, (size_t)jb.W * jb.nb * 4 * jb.h->F * 4, sw.st));
    }
    const bool history = sw.jobs[0].h->ws.history != 0;
    auto store_ckpt = [&](int n) -> probe_status {
        if (!ckpt || history || n % sw.K) return PROBE_OK;
        for (Job& jb : sw.jobs) {
            Workspace& w = jb.h->ws;
            const int k = n / sw.K;
            const size_t per = (size_t)jb.W * ckpt_bytes_per_shot(jb.h->snap, jb.h->F);
            cudaError_t e = launch_encode_ckpt(w.u4, jb.W * 2, jb.h->F, 4, n & 3, (n + 3) & 3, (char*)w.ckpt + k * per,
                                               w.scales + (size_t)k * jb.W * 2, jb.h->snap, w.absmax, sw.st);
            if (e != cudaSuccess) return cuda_fail(jb.h, e, "checkpoint store");
            sw.launches_other += codec_launches(jb.h->snap, true, 4, n & 3);
        }
        return PROBE_OK;
    };
    for (int n = 0; n < sw.nt - 1;) {
        const bool two = n + 2 <= sw.nt - 1;
        TRY(store_ckpt(n));
        TRY(launch_fwd_tb(sw, FWD_BORN, n, two, history ? n : 0));
        sw.launches_fwd++;
        if (two) TRY(store_ckpt(n + 1));
        n += two ? 2 : 1;
    }
    const int plane = (sw.nt - 1) & 3;  // last time level at the receivers
    for (Job& jb : sw.jobs) {
        probe_t h = jb.h;
        Workspace& w = h->ws;
        cudaError_t e = launch_sample(w.f4, (long long)jb.nb * 4 * h->F, 4 * h->F, plane, h->F, jb.W, jb.nb, h->d_rec,
                                      h->nr, h->P, h->ndim, h->Ny, jb.data, jb.dss, jb.dts, sw.nt - 1, sw.st);
        if (e != cudaSuccess) return cuda_fail(h, e, "receiver sampling");
        sw.launches_other++;
    }
    return PROBE_OK;
}

probe_status run_forward(Sweep& sw, FwdKind kind, bool ckpt) {
    if (sw.tb == 2 && kind == FWD_BORN) return run_forward_tb(sw, ckpt);
    for (Job& jb : sw.jobs) {
        Workspace& w = jb.h->ws;
        CK(jb.h, cudaMemsetAsync(w.u, 0, (size_t)jb.W * 2 * jb.h->F * 4, sw.st));
        if (kind == FWD_BORN)
            CK(jb.h, cudaMemsetAsync(w.f, 0, (size_t)jb.W * jb.nb * 2 * jb.h->F * 4, sw.st));
    }
    const bool history = sw.jobs[0].h->ws.history != 0;
    if (history && kind == FWD_INCIDENT) kind = FWD_INCIDENT_DTT;  // Dtt u^n of every step
    for (int n = 0; n < sw.nt - 1; ++n) {
        if (ckpt && !history && n % sw.K == 0) {
            for (Job& jb : sw.jobs) {
                Workspace& w = jb.h->ws;
                const int k = n / sw.K;
                const size_t per = (size_t)jb.W * ckpt_bytes_per_shot(jb.h->snap, jb.h->F);
                void* dst = (char*)w.ckpt + (size_t)k * per;
                cudaError_t e = launch_encode_ckpt(w.u, jb.W * 2, jb.h->F, 2, n & 1, (n & 1) ^ 1, dst,
                                                   w.scales + (size_t)k * jb.W * 2, jb.h->snap, w.absmax, sw.st);
                if (e != cudaSuccess) return cuda_fail(jb.h, e, "checkpoint store");
                sw.launches_other += codec_launches(jb.h->snap, true, 2, n & 1);
            }
        }
        TRY(launch_fwd_step(sw, kind, n, history ? n : 0));
        sw.launches_fwd++;
    }
    // last time level at the receivers
    if (kind == FWD_BORN || kind == FWD_INCIDENT_SAMPLE) {
        const int plane = (sw.nt - 1) & 1;
        for (Job& jb : sw.jobs) {
            probe_t h = jb.h;
            Workspace& w = h->ws;
            const bool born = kind == FWD_BORN;
            cudaError_t e = launch_sample(born ? w.f : w.u, (long long)(born ? jb.nb : 1) * 2 * h->F,
                                          2 * h->F, plane, h->F, jb.W, born ? jb.nb : 1, h->d_rec, h->nr,
                                          h->P, h->ndim, h->Ny, jb.data, jb.dss, jb.dts, sw.nt - 1, sw.st);
            if (e != cudaSuccess) return cuda_fail(h, e, "receiver sampling");
            sw.launches_other++;
        }
    }
    return PROBE_OK;
}

// Adjoint sweep with segment-wise recomputation; accumulates into the images.
// Receiver injection R^T r^n of time levels n_hi down to n_lo for every model of the sweep,
// into the segment buffer (slot k = level n_hi - k); the adjoint steps read it.
probe_status build_injection(Sweep& sw, int n_hi, int n_lo) {
    for (Job& jb : sw.jobs) {
        probe_t h = jb.h;
        Workspace& w = h->ws;
        if (!w.inj || h->nband == 0) continue;
        const long long block = inj_block(h);
        const int nb = std::max(jb.nb, 1);
        CK(h, cudaMemsetAsync(w.inj, 0, (size_t)(n_hi - n_lo + 1) * jb.W * nb * block * 4, sw.st));
        cudaError_t e = launch_build_injection(jb.rdata, jb.dss, jb.dts, h->nr, n_hi, n_hi - n_lo + 1, jb.W, nb,
                                               h->nuc, h->d_uc_ptr, h->d_uc_rec, h->d_uc_pos, w.inj, block, sw.st);
        if (e != cudaSuccess) return cuda_fail(h, e, "receiver injection");
        sw.launches_other++;
    }
    sw.inj_hi = n_hi;
    return PROBE_OK;
}

probe_status run_adjoint(Sweep& sw) {
    for (Job& jb : sw.jobs) {
        Workspace& w = jb.h->ws;
        CK(jb.h, cudaMemsetAsync(w.f, 0, (size_t)jb.W * jb.nb * 2 * jb.h->F * 4, sw.st));
    }
    probe_t h0 = sw.jobs[0].h;
    int ev = 2;
    if (h0->ws.history) {  // Dtt u^n kept for every step: no recomputation
        record(h0, ev++, sw.st);
        record(h0, ev++, sw.st);
        for (int n_hi = sw.nt - 1; n_hi >= 1; n_hi -= sw.K) {  // injection built K levels at a time
            const int n_lo = std::max(1, n_hi - sw.K + 1);
            TRY(build_injection(sw, n_hi, n_lo));
            for (int n = n_hi; n >= n_lo; --n) {
                TRY(launch_adj_step(sw, n, n - 1));
                sw.launches_adj += sw.chunks;
            }
        }
        record(h0, ev++, sw.st);
        return PROBE_OK;
    }
    for (int k = sw.nck - 1; k >= 0; --k) {
        const int k0 = k * sw.K;
        const int k1 = std::min(k0 + sw.K, sw.nt - 1);
        if (k0 >= k1) continue;
        record(h0, ev++, sw.st);
        const bool tb = sw.tb == 2;  // recompute two levels per launch over the four-level state
        for (Job& jb : sw.jobs) {
            Workspace& w = jb.h->ws;
            const size_t per = (size_t)jb.W * ckpt_bytes_per_shot(jb.h->snap, jb.h->F);
            const void* src = (const char*)w.ckpt + (size_t)k * per;
            cudaError_t e = tb ? launch_decode_ckpt(src, w.scales + (size_t)k * jb.W * 2, jb.W * 2, jb.h->F, 4, k0 & 3,
                                                    (k0 + 3) & 3, jb.h->snap, w.u4, sw.st)
                               : launch_decode_ckpt(src, w.scales + (size_t)k * jb.W * 2, jb.W * 2, jb.h->F, 2, k0 & 1,
                                                    (k0 & 1) ^ 1, jb.h->snap, w.u, sw.st);
            if (e != cudaSuccess) return cuda_fail(jb.h, e, "checkpoint restore");
            sw.launches_other += tb ? codec_launches(jb.h->snap, false, 4, k0 & 3)
                                    : codec_launches(jb.h->snap, false, 2, k0 & 1);
        }
        if (tb) {
            for (int j = k0; j < k1;) {
                const bool two = j + 2 <= k1;
                TRY(launch_fwd_tb(sw, FWD_INCIDENT_DTT, j, two, j - k0));
                sw.launches_rec++;
                j += two ? 2 : 1;
            }
        } else {
            for (int j = k0; j < k1; ++j) {
                TRY(launch_fwd_step(sw, FWD_INCIDENT_DTT, j, j - k0));
                sw.launches_rec++;
            }
        }
        record(h0, ev++, sw.st);
        TRY(build_injection(sw, k1, k0 + 1));
        for (int n = k1; n >= k0 + 1; --n) {
            TRY(launch_adj_step(sw, n, n - 1 - k0));
            sw.launches_adj += sw.chunks;
        }
    }
    record(h0, ev++, sw.st);
    return PROBE_OK;
}

// ---------------------------------------------------------------------------
// 3D sweeps: one launch per field kind and step (incident, Born trials, adjoint).
// ---------------------------------------------------------------------------
long long dtt_stride3(probe_t h) { return (long long)(h->ws.with_ckpt ? h->K : 2) * h->F; }

void fill3d(const Job& jb, ModelStep3D& m) {
    probe_t h = jb.h;
    Workspace& w = h->ws;
    memset(&m, 0, sizeof(m));
    m.Nz = h->Nz;
    m.Ny = h->Ny;
    m.Nx = h->Nx;
    m.P = h->P;
    m.pad = h->pad;
    m.nz = h->nz;
    m.ny = h->ny;
    m.nx = h->nx;
    m.tiles_x = h->tiles_x;
    m.tiles_y = h->tiles_y;
    m.zchunks = (h->Nz + h->zc3d - 1) / h->zc3d;
    m.ZC = h->zc3d;
    m.nshots = jb.W;
    m.nr = h->nr;
    m.cz = h->cz;
    m.cy = h->cy;
    m.cx = h->cx;
    const double wk[4] = {PROBE_W1, PROBE_W2, PROBE_W3, PROBE_W4};
    for (int k = 0; k < 4; ++k) {
        m.lz[k] = (float)(wk[k] / (h->hz * h->hz));
        m.ly[k] = (float)(wk[k] / (h->hy * h->hy));
        m.lx[k] = (float)(wk[k] / (h->hx * h->hx));
    }
    for (int mm = 0; mm < 4; ++mm) {  // first-difference x taps: sum_{k>m} w_k / hx^2
        double cm = 0.0;
        for (int k = mm; k < 4; ++k) cm += wk[k];
        m.cxm[mm] = (float)(cm / (h->hx * h->hx));
    }
    m.inv_dt2 = (float)(1.0 / (h->dt * h->dt));
    m.vol_inv = (float)(1.0 / (h->hz * h->hy * h->hx));
    m.F = h->F;
    m.s = jb.s;
    m.dm = w.dm;
    m.wavelet = h->d_wavelet;
    m.src = w.src_wave;
    m.rec_ptr = h->d_rec_tile_ptr;
    m.rec_idx = h->d_rec_tile_idx;
    m.rec_zyx = h->d_rec;
    m.data = jb.data;
    m.rdata = jb.rdata;
    m.dss = jb.dss;
    m.dts = jb.dts;
    m.img = w.img;
    m.comp = w.comp;
}

struct Count3 {
    long long fwd = 0, rec = 0, adj = 0, other = 0;
};

probe_status launch3(probe_t h, int mode, StepParams3D& p, int n, cudaStream_t st, const char* what) {
    p.n = n;
    // the incident step (forward and recompute) may use its own ring-refill scheme
    const int pipe = (mode == STEP3_INC || mode == STEP3_INC_SAMPLE) ? h->pipe_inc : h->opt_pipeline;
    cudaError_t e = launch_step3d(mode, h->kahan != 0, pipe, p, st);
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    return PROBE_OK;
}

// 3D autotuner, on the first call for a workload key, timed on the real workspace (round-robin
// over three rounds, each candidate's fastest round kept): the z planes one CTA marches (32, 64,
// 128) with the ring-refill scheme of the pipelined forward kernels (2: producer warp, 3: the
// last compute warp out of a slot) on one incident and (for the Born forward) one Born launch per
// candidate; then, for calls with an adjoint sweep, the refill scheme of the adjoint on one
// adjoint launch per scheme.  The launches write only the state planes, the Dtt plane and the
// segment image or the image, which the call clears or rewrites before it reads them.  None of
// the choices changes a result.
probe_status autotune_3d(const Job& jb, FwdKind kind, bool adjoint, cudaStream_t st) {
    probe_t h = jb.h;
    const bool fam_fixed = h->user_fixed || h->opt_pipeline == 0;
    if (h->ndim != 3 || (h->user_zc3d && fam_fixed) || h->opt_cluster3d) return PROBE_OK;
    const std::vector<long long> key = {(long long)kind, (long long)adjoint, jb.W, jb.nb};
    for (const Tuned3& t : h->tuned3)
        if (t.key == key) {
            if (!h->user_zc3d) h->zc3d = t.zc;
            if (!fam_fixed) {
                h->opt_pipeline = t.fam_fwd;
                h->pipe_inc = t.fam_inc;
                h->pipe_adj = t.fam_adj;
            }
            return PROBE_OK;
        }
    if (!h->opt_autotune) return PROBE_OK;
    Workspace& w = h->ws;
    if (!w.dtt) return PROBE_OK;
    const bool born = kind == FWD_BORN;
    StepParams3D pi, pb, pa;
    fill3d(jb, pi.m);
    pi.nt = h->nt;
    pi.err = h->d_err;
    pi.m.tm = w.tm_u;
    pi.m.state = w.u;
    pi.m.nfield = 1;
    pi.m.nvol_shot = 2;
    pi.m.Dout = w.dtt;
    pi.m.Dout_shot_stride = dtt_stride3(h);
    fill3d(jb, pb.m);  // Born fields (forward) and adjoint fields share the f planes
    pb.nt = h->nt;
    pb.err = h->d_err;
    pb.m.tm = w.tm_f;
    pb.m.state = w.f;
    pb.m.nfield = jb.nb;
    pb.m.nvol_shot = 2 * jb.nb;
    pb.m.Din = w.dtt;
    pb.m.Din_shot_stride = dtt_stride3(h);
    pa = pb;  // adjoint: no receiver injection (rrow null); a segment's first step writes its image
    if (w.seg) {
        pa.m.img = w.seg;
        pa.m.seg_first = 1;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(h, ce, "autotuner events");
    }
    // times `body` (which launches on st) and keeps the minimum in *best
    auto timed = [&](float* best, auto body) -> probe_status {
        cudaEventRecord(e0, st);
        probe_status ps = body();
        cudaEventRecord(e1, st);
        if (ps != PROBE_OK) return ps;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return cuda_fail(h, e, "autotuner timing");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *best = std::min(*best, ms);
        return PROBE_OK;
    };
    auto set_zc = [&](int zc) {
        for (StepParams3D* q : {&pi, &pb, &pa}) {
            q->m.ZC = zc;
            q->m.zchunks = (h->Nz + zc - 1) / zc;
        }
    };
    // forward: (refill scheme, planes), the incident and the Born launches timed apart so that
    // each gets its own scheme; the caller's fixed choices stay fixed
    std::vector<int> fams = {2, 3}, zcs = {32, 64, 128};
    if (fam_fixed) fams = {h->opt_pipeline};
    if (h->user_zc3d) zcs = {h->zc3d};
    std::vector<std::pair<int, int>> cand;
    for (int fam : fams)
        for (int zc : zcs) cand.push_back({fam, zc});
    const int nc = (int)cand.size();
    std::vector<float> t_inc(nc, 1e30f), t_born(nc, born ? 1e30f : 0.f);
    probe_status ps = PROBE_OK;
    for (int round = 0; round < 3 && ps == PROBE_OK; ++round)
        for (int c = 0; c < nc && ps == PROBE_OK; ++c) {
            set_zc(cand[c].second);
            for (int mode : {STEP3_INC, STEP3_BORN}) {
                if (ps != PROBE_OK || (mode == STEP3_BORN && !born)) continue;
                StepParams3D& q = (mode == STEP3_INC) ? pi : pb;
                ps = timed(mode == STEP3_INC ? &t_inc[c] : &t_born[c], [&]() -> probe_status {
                    for (int n = 0; n < 2; ++n) {
                        q.n = n;
                        cudaError_t e = launch_step3d(mode, false, cand[c].first, q, st);
                        if (e != cudaSuccess) return cuda_fail(h, e, "autotuner launch");
                    }
                    return PROBE_OK;
                });
            }
        }
    // per plane count the faster scheme of each launch; then the plane count of the fastest step
    int zc = h->zc3d, fam_inc = fams[0], fam_fwd = fams[0];
    float best_step = 1e30f;
    for (int z : zcs) {
        int bi = -1, bb = -1;
        for (int c = 0; c < nc; ++c) {
            if (cand[c].second != z) continue;
            if (bi < 0 || t_inc[c] < t_inc[bi]) bi = c;
            if (bb < 0 || t_born[c] < t_born[bb]) bb = c;
        }
        if (bi >= 0 && t_inc[bi] + t_born[bb] < best_step) {
            best_step = t_inc[bi] + t_born[bb];
            zc = z;
            fam_inc = cand[bi].first;
            fam_fwd = cand[bb].first;
        }
    }
    // adjoint refill scheme at the chosen planes
    int fam_adj = fam_fixed ? h->pipe_adj : fam_fwd;
    if (ps == PROBE_OK && adjoint && !fam_fixed && adj3d_ws(h)) {
        float ba[2] = {1e30f, 1e30f};
        set_zc(zc);
        for (int round = 0; round < 3 && ps == PROBE_OK; ++round)
            for (int c = 0; c < 2 && ps == PROBE_OK; ++c)
                ps = timed(&ba[c], [&]() -> probe_status {
                    for (int n = 0; n < 2; ++n) {
                        pa.n = h->nt - 1 - n;
                        cudaError_t e = launch_step3d(STEP3_ADJ, false, 2 + c, pa, st);
                        if (e != cudaSuccess) return cuda_fail(h, e, "autotuner launch");
                    }
                    return PROBE_OK;
                });
        fam_adj = (ba[1] < ba[0]) ? 3 : 2;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TRY(ps);
    h->zc3d = zc;
    if (!fam_fixed) {
        h->opt_pipeline = born ? fam_fwd : fam_inc;
        h->pipe_inc = fam_inc;
        h->pipe_adj = fam_adj;
    }
    Tuned3 t;
    t.key = key;
    t.fam_fwd = h->opt_pipeline;
    t.fam_inc = h->pipe_inc;
    t.fam_adj = h->pipe_adj;
    t.zc = h->zc3d;
    h->tuned3.push_back(t);
    return PROBE_OK;
}

probe_status ensure_overlap_stream(probe_t h) {
    if (h->ostream) return PROBE_OK;
    CK(h, cudaStreamCreateWithFlags(&h->ostream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        CK(h, cudaEventCreateWithFlags(&h->ov_inc[i], cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ov_born[i], cudaEventDisableTiming));
    }
    return PROBE_OK;
}

probe_status run_forward3d(const Job& jb, FwdKind kind, bool ckpt, cudaStream_t st, Count3& c) {
    probe_t h = jb.h;
    Workspace& w = h->ws;
    const bool born = kind == FWD_BORN;
    CK(h, cudaMemsetAsync(w.u, 0, (size_t)jb.W * 2 * h->F * 4, st));
    if (born) CK(h, cudaMemsetAsync(w.f, 0, (size_t)jb.W * jb.nb * 2 * h->F * 4, st));
    StepParams3D pi, pb;
    fill3d(jb, pi.m);
    pi.nt = h->nt;
    pi.err = h->d_err;
    pi.m.tm = w.tm_u;
    pi.m.state = w.u;
    pi.m.nfield = 1;
    pi.m.nvol_shot = 2;
    pi.m.Dout = born ? w.dtt : nullptr;
    pi.m.Dout_shot_stride = dtt_stride3(h);
    if (born) {
        fill3d(jb, pb.m);
        pb.nt = h->nt;
        pb.err = h->d_err;
        pb.m.tm = w.tm_f;
        pb.m.state = w.f;
        pb.m.nfield = jb.nb;
        pb.m.nvol_shot = 2 * jb.nb;
        pb.m.Din = w.dtt;
        pb.m.Din_shot_stride = dtt_stride3(h);
    }
    const int imode = (kind == FWD_INCIDENT_SAMPLE) ? STEP3_INC_SAMPLE : STEP3_INC;
    // fused incident + Born step on thread-block clusters (Dtt u0 exchanged in shared memory)
    const bool fused = born && (h->opt_cluster3d & 1) && jb.nb + 1 <= 8;
    StepParams3D pf;
    if (fused) {
        pf.nt = h->nt;
        pf.err = h->d_err;
        pf.m = pi.m;
        pf.m.Dout = nullptr;
        pf.m2 = pb.m;
        pf.m2.Din = nullptr;
    }
    // overlapped forward: the incident step n writes Dtt u^n into slot n & 1 on `st`; the Born
    // step n reads it on the second stream after the incident step's event, and the incident step
    // n + 2 (the slot's next writer) waits for the Born step n's event.  Both streams are joined
    // to `st` before the sampling.
    const bool overlap = born && !fused && h->opt_overlap3d && w.dtt_slots >= 2;
    if (overlap) TRY(ensure_overlap_stream(h));
    cudaStream_t sb = overlap ? h->ostream : st;
    if (overlap) {  // the Born stream starts after everything queued on st so far
        CK(h, cudaEventRecord(h->ov_inc[0], st));
        CK(h, cudaStreamWaitEvent(sb, h->ov_inc[0], 0));
    }
    for (int n = 0; n < h->nt - 1; ++n) {
        if (ckpt && n % h->K == 0) {
            const int k = n / h->K;
            const size_t per = (size_t)jb.W * ckpt_bytes_per_shot(h->snap, h->F);
            void* dst = (char*)w.ckpt + (size_t)k * per;
            cudaError_t e = launch_encode_ckpt(w.u, jb.W * 2, h->F, 2, n & 1, (n & 1) ^ 1, dst,
                                               w.scales + (size_t)k * jb.W * 2, h->snap, w.absmax, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint store");
            c.other += codec_launches(h->snap, true, 2, n & 1);
        }
        if (fused) {
            pf.n = n;
            cudaError_t e = launch_fwd3d_cluster(pf, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "fused forward step launch");
            c.fwd++;
            continue;
        }
        const int slot = overlap ? (n & 1) : 0;
        if (overlap && n >= 2) CK(h, cudaStreamWaitEvent(st, h->ov_born[slot], 0));
        if (born) pi.m.Dout = w.dtt + (long long)slot * h->F;
        TRY(launch3(h, imode, pi, n, st, "incident step launch"));
        c.fwd++;
        if (born) {
            if (overlap) {
                CK(h, cudaEventRecord(h->ov_inc[slot], st));
                CK(h, cudaStreamWaitEvent(sb, h->ov_inc[slot], 0));
            }
            pb.m.Din = w.dtt + (long long)slot * h->F;
            TRY(launch3(h, STEP3_BORN, pb, n, sb, "Born step launch"));
            if (overlap) CK(h, cudaEventRecord(h->ov_born[slot], sb));
            c.fwd++;
        }
    }
    if (overlap) {  // join the Born stream back into st
        CK(h, cudaEventRecord(h->ov_born[0], sb));
        CK(h, cudaStreamWaitEvent(st, h->ov_born[0], 0));
    }
    if (born || kind == FWD_INCIDENT_SAMPLE) {
        cudaError_t e = launch_sample(born ? w.f : w.u, (long long)(born ? jb.nb : 1) * 2 * h->F, 2 * h->F,
                                      (h->nt - 1) & 1, h->F, jb.W, born ? jb.nb : 1, h->d_rec, h->nr, h->P, 3,
                                      h->Ny, jb.data, jb.dss, jb.dts, h->nt - 1, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "receiver sampling");
        c.other++;
    }
    return PROBE_OK;
}

probe_status run_adjoint3d(const Job& jb, cudaStream_t st, Count3& c) {
    probe_t h = jb.h;
    Workspace& w = h->ws;
    CK(h, cudaMemsetAsync(w.f, 0, (size_t)jb.W * jb.nb * 2 * h->F * 4, st));
    StepParams3D pi, pa;
    fill3d(jb, pi.m);
    pi.nt = h->nt;
    pi.err = h->d_err;
    pi.m.tm = w.tm_u;
    pi.m.state = w.u;
    pi.m.nfield = 1;
    pi.m.nvol_shot = 2;
    pi.m.Dout_shot_stride = dtt_stride3(h);
    fill3d(jb, pa.m);
    pa.nt = h->nt;
    pa.err = h->d_err;
    pa.m.tm = w.tm_f;
    pa.m.state = w.f;
    pa.m.nfield = jb.nb;
    pa.m.nvol_shot = 2 * jb.nb;
    pa.m.Din_shot_stride = dtt_stride3(h);
    // shot-cluster adjoint: images of shot groups summed in shared memory, receiver injection
    // prebuilt per segment for the planes that hold receivers
    const bool clustered = (h->opt_cluster3d & 2) != 0;
    // producer-warp adjoint: needs the injection buffer wherever there are receivers (a workspace
    // sized before the option was set has none; the one-barrier kernel then assembles it itself)
    const bool ws = adj3d_ws(h) && (h->nband == 0 || w.inj != nullptr);
    const int G = pick_group(h, h->ws.W);
    const long long block = inj_block(h);
    if (clustered || ws) {
        pa.m.rrow = (h->nband > 0) ? h->d_rrow : nullptr;
        pa.m.inj = (h->nband > 0) ? w.inj : nullptr;
        pa.m.inj_block = block;
    }
    int ev = 2;
    for (int k = h->nck - 1; k >= 0; --k) {
        const int k0 = k * h->K;
        const int k1 = std::min(k0 + h->K, h->nt - 1);
        if (k0 >= k1) continue;
        record(h, ev++, st);
        const size_t per = (size_t)jb.W * ckpt_bytes_per_shot(h->snap, h->F);
        const void* src = (const char*)w.ckpt + (size_t)k * per;
        cudaError_t e = launch_decode_ckpt(src, w.scales + (size_t)k * jb.W * 2, jb.W * 2, h->F, 2, k0 & 1,
                                           (k0 & 1) ^ 1, h->snap, w.u, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint restore");
        c.other += codec_launches(h->snap, false, 2, k0 & 1);
        for (int j = k0; j < k1; ++j) {
            pi.m.Dout = w.dtt + (long long)(j - k0) * h->F;
            TRY(launch3(h, STEP3_INC, pi, j, st, "recompute step launch"));
            c.rec++;
        }
        record(h, ev++, st);
        if ((clustered || ws) && h->nband > 0) {  // R^T r^n of levels k1 .. k0 + 1, slot k1 - n
            CK(h, cudaMemsetAsync(w.inj, 0, (size_t)(k1 - k0) * jb.W * jb.nb * block * 4, st));
            cudaError_t e = launch_build_injection(jb.rdata, jb.dss, jb.dts, h->nr, k1, k1 - k0, jb.W, jb.nb, h->nuc,
                                                   h->d_uc_ptr, h->d_uc_rec, h->d_uc_pos, w.inj, block, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "receiver injection");
            c.other++;
        }
        for (int n = k1; n >= k0 + 1; --n) {
            pa.m.Din = w.dtt + (long long)(n - 1 - k0) * h->F;
            if (clustered) {
                pa.n = n;
                pa.m.inj_slot = k1 - n;
                cudaError_t e = launch_adj3d_cluster(G, h->kahan != 0, pa, st);
                if (e != cudaSuccess) return cuda_fail(h, e, "adjoint step launch");
            } else {
                // with Kahan compensation: two-level imaging sum, plain FP32 within the segment,
                // Kahan across segments; without: plain FP32 into the image itself
                pa.n = n;
                pa.m.inj_slot = k1 - n;
                if (w.seg) {
                    pa.m.img = w.seg;
                    pa.m.seg_first = (n == k1) ? 1 : 0;
                }
                cudaError_t e = launch_step3d(STEP3_ADJ, !w.seg && h->kahan != 0, ws ? h->pipe_adj : 0, pa, st);
                if (e != cudaSuccess) return cuda_fail(h, e, "adjoint step launch");
            }
            c.adj++;
        }
        if (w.seg) {
            cudaError_t e = launch_kahan_fold(w.img, w.comp, w.seg, (long long)jb.W * jb.nb * h->F, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "segment image fold");
            c.other++;
        }
    }
    record(h, ev++, st);
    return PROBE_OK;
}

probe_status check_dev_error(probe_t h, cudaStream_t st) {
    CK(h, cudaStreamSynchronize(st));
    int e = 0;
    CK(h, cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        CK(h, cudaMemset(h->d_err, 0, sizeof(int)));
        if (e & DEVERR_TIMEOUT) return fail(h, PROBE_ERR_TIMEOUT, "a bounded device wait timed out");
        if (e & DEVERR_NONFINITE) return fail(h, PROBE_ERR_NONFINITE, "NaN or Inf in an input or output");
    }
    return PROBE_OK;
}

void clear_graphs(probe_t h) {
    for (GraphEntry& g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

probe_status ensure_graph_stream(probe_t h) {
    if (h->gstream) return PROBE_OK;
    CK(h, cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    CK(h, cudaEventCreateWithFlags(&h->gev_in, cudaEventDisableTiming));
    CK(h, cudaEventCreateWithFlags(&h->gev_out, cudaEventDisableTiming));
    return PROBE_OK;
}

// Run `body(stream)` for one wave either eagerly on `st` or as a cached CUDA graph
// (captured once per key on the library stream and replayed there, joined to `st`
// by events).
template <typename Body>
probe_status run_maybe_graph(probe_t h, const std::vector<long long>& key, cudaStream_t st, long long counts[4],
                             Body body) {
    if (!h->opt_use_graph) return body(st);  // timing events are captured as event-record nodes
    TRY(ensure_graph_stream(h));
    if (h->graph_generation != h->ws.generation) {
        clear_graphs(h);
        h->graph_generation = h->ws.generation;
    }
    cudaGraphExec_t exec = nullptr;
    for (GraphEntry& g : h->graphs)
        if (g.key == key) {
            exec = g.exec;
            for (int i = 0; i < 4; ++i) counts[i] = g.counts[i];
        }
    if (!exec) {
        CK(h, cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal));
        probe_status s = body(h->gstream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->gstream, &graph);
        if (s != PROBE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
        if (h->graphs.size() >= 16) {
            cudaGraphExecDestroy(h->graphs.front().exec);
            h->graphs.erase(h->graphs.begin());
        }
        GraphEntry g;
        g.key = key;
        g.exec = exec;
        for (int i = 0; i < 4; ++i) g.counts[i] = counts[i];
        h->graphs.push_back(g);
    }
    CK(h, cudaEventRecord(h->gev_in, st));
    CK(h, cudaStreamWaitEvent(h->gstream, h->gev_in, 0));
    CK(h, cudaGraphLaunch(exec, h->gstream));
    CK(h, cudaEventRecord(h->gev_out, h->gstream));
    CK(h, cudaStreamWaitEvent(st, h->gev_out, 0));
    return PROBE_OK;
}

// Stage an input array on the device (returns a device pointer).
probe_status stage_input(probe_t h, const float* p, size_t n, DevBuf& buf, const float** out,
                         cudaStream_t st, bool* was_host) {
    *was_host = false;
    if (is_device_ptr(p)) {
        *out = p;
        return PROBE_OK;
    }
    *was_host = true;
    TRY(ensure_buf(h, buf, n * 4));
    CK(h, cudaMemcpyAsync(buf.p, p, n * 4, cudaMemcpyHostToDevice, st));
    *out = (const float*)buf.p;
    return PROBE_OK;
}

void reset_stats(probe_t h) {
    h->stats = probe_stats();
    h->stats.ckpt_stride = h->K;
    h->stats.tile_z = h->tile_z;
    h->stats.dtt_history = h->ws.history;
}

void finish_stats(probe_t h, const Sweep& sw, int nwaves_events) {
    (void)nwaves_events;
    probe_stats& s = h->stats;
    s.launches_forward += sw.launches_fwd;
    s.launches_recompute += sw.launches_rec;
    s.launches_adjoint += sw.launches_adj;
    s.launches_total += sw.launches_fwd + sw.launches_rec + sw.launches_adj + sw.launches_other;
}


}  // namespace

// ---------------------------------------------------------------------------
// Handle creation
// ---------------------------------------------------------------------------
extern "C" probe_status probe_create(probe_t* out, const probe_grid* g, const float* m0, int ns,
                                     const int* src_idx, int nr, const int* rec_idx,
                                     const float* wavelet, int nt, double dt) {
    if (!out) return fail(nullptr, PROBE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !m0 || !src_idx || !rec_idx || !wavelet)
        return fail(nullptr, PROBE_ERR_ARG, "NULL argument");
    if (g->ndim != 2 && g->ndim != 3) return fail(nullptr, PROBE_ERR_ARG, "ndim must be 2 or 3");
    for (int a = 0; a < g->ndim; ++a) {
        if (g->n[a] < 1 || g->n[a] > (1 << 20)) return fail(nullptr, PROBE_ERR_ARG, "grid size out of range");
        if (!(g->h[a] > 0) || !std::isfinite(g->h[a])) return fail(nullptr, PROBE_ERR_ARG, "spacing must be > 0");
    }
    if (g->pad < 0 || g->pad > 4096) return fail(nullptr, PROBE_ERR_ARG, "pad out of range");
    if (g->snapshot_dtype < 0 || g->snapshot_dtype > 2)
        return fail(nullptr, PROBE_ERR_ARG, "snapshot_dtype must be 0, 1 or 2");
    if (g->ckpt_stride < 0) return fail(nullptr, PROBE_ERR_ARG, "ckpt_stride must be >= 0");
    if (ns < 1 || nr < 1 || nt < 2) return fail(nullptr, PROBE_ERR_ARG, "need ns >= 1, nr >= 1, nt >= 2");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(nullptr, PROBE_ERR_ARG, "dt must be > 0");

    probe_t h = new probe_s();
    const int D = g->ndim;
    h->ndim = D;
    h->nz = g->n[0];
    h->ny = D == 3 ? g->n[1] : 1;
    h->nx = g->n[D - 1];
    h->hz = g->h[0];
    h->hy = D == 3 ? g->h[1] : 1.0;
    h->hx = g->h[D - 1];
    h->pad = g->pad;
    h->Nz = h->nz + 2 * h->pad;
    h->Ny = D == 3 ? h->ny + 2 * h->pad : 1;
    h->Nx = h->nx + 2 * h->pad;
    h->P = ((h->Nx + 31) / 32) * 32;
    h->F = (long long)h->Nz * h->Ny * h->P;
    h->nmodel = (long long)h->nz * h->ny * h->nx;
    h->dt = dt;
    h->nt = nt;
    h->ns = ns;
    h->nr = nr;
    h->snap = g->snapshot_dtype;
    h->kahan = g->kahan ? 1 : 0;
    h->K = g->ckpt_stride > 0 ? g->ckpt_stride : (int)std::ceil(std::sqrt((double)nt));
    h->K = std::max(1, std::min(h->K, nt - 1));
    h->nck = (nt - 2) / h->K + 1;  // checkpoints at n = 0, K, ... < nt - 1

    auto bad = [&](const std::string& m) {
        probe_destroy(h);
        return fail(nullptr, PROBE_ERR_ARG, m);
    };
    // indices (padded copies kept in the same (z[, y], x) order)
    h->src_pad.resize((size_t)ns * D);
    h->rec_pad.resize((size_t)nr * D);
    std::vector<int> sidx((size_t)ns * D), ridx((size_t)nr * D);
    if (is_device_ptr(src_idx)) {
        if (cudaMemcpy(sidx.data(), src_idx, sidx.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return bad("cannot read src_idx");
    } else
        memcpy(sidx.data(), src_idx, sidx.size() * 4);
    if (is_device_ptr(rec_idx)) {
        if (cudaMemcpy(ridx.data(), rec_idx, ridx.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return bad("cannot read rec_idx");
    } else
        memcpy(ridx.data(), rec_idx, ridx.size() * 4);
    const int nlim[3] = {h->nz, D == 3 ? h->ny : h->nx, h->nx};
    for (int s = 0; s < ns; ++s)
        for (int a = 0; a < D; ++a) {
            const int v = sidx[(size_t)D * s + a];
            if (v < 0 || v >= nlim[a]) return bad("source index outside the interior");
            h->src_pad[(size_t)D * s + a] = v + h->pad;
        }
    for (int r = 0; r < nr; ++r)
        for (int a = 0; a < D; ++a) {
            const int v = ridx[(size_t)D * r + a];
            if (v < 0 || v >= nlim[a]) return bad("receiver index outside the interior");
            h->rec_pad[(size_t)D * r + a] = v + h->pad;
        }
    // model: positivity, finiteness, CFL
    std::vector<float> m0h((size_t)h->nmodel);
    std::vector<float> wh((size_t)nt);
    if (is_device_ptr(m0)) {
        if (cudaMemcpy(m0h.data(), m0, m0h.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return bad("cannot read m0");
    } else
        memcpy(m0h.data(), m0, m0h.size() * 4);
    if (is_device_ptr(wavelet)) {
        if (cudaMemcpy(wh.data(), wavelet, wh.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return bad("cannot read wavelet");
    } else
        memcpy(wh.data(), wavelet, wh.size() * 4);
    float mmin = INFINITY;
    for (float v : m0h) {
        if (!std::isfinite(v) || !(v > 0)) {
            probe_destroy(h);
            return fail(nullptr, PROBE_ERR_NONFINITE, "m0 must be finite and > 0");
        }
        mmin = std::min(mmin, v);
    }
    for (float v : wh)
        if (!std::isfinite(v)) {
            probe_destroy(h);
            return fail(nullptr, PROBE_ERR_NONFINITE, "wavelet must be finite");
        }
    h->cmax = 1.0 / std::sqrt((double)mmin);
    const double hmin = std::min(h->hz, std::min(h->hx, D == 3 ? h->hy : h->hx));
    // leapfrog + 8th-order Laplacian: c dt / h < 2 / sqrt(D * (|w0| + 2 sum |w_k|))
    const double limit = 2.0 / std::sqrt(D * (205.0 / 72.0 + 2 * (8.0 / 5 + 1.0 / 5 + 8.0 / 315 + 1.0 / 560)));
    if (h->cmax * dt / hmin >= limit) {
        char buf[160];
        snprintf(buf, sizeof buf, "CFL violated: c_max dt / h_min = %.4f >= %.4f", h->cmax * dt / hmin, limit);
        return bad(buf);
    }
    // sponge: eta dt/2 = (dt/2) eta_max (rho/pad)^2 per axis
    if (h->pad > 0) {
        const double R = 1e-3;
        auto coef = [&](double ha) {
            const double em = 3.0 * h->cmax * std::log(1.0 / R) / (2.0 * h->pad * ha);
            return (float)(0.5 * dt * em / ((double)h->pad * h->pad));
        };
        h->cz = coef(h->hz);
        h->cx = coef(h->hx);
        h->cy = D == 3 ? coef(h->hy) : 0.f;
    }

    auto cuda_bad = [&](cudaError_t e, const char* what) {
        std::string m = std::string(what) + ": " + cudaGetErrorString(e);
        probe_destroy(h);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? PROBE_ERR_OOM : PROBE_ERR_CUDA, m);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&h->d_m0, m0h.size() * 4)) != cudaSuccess) return cuda_bad(e, "alloc m0");
    if ((e = cudaMemcpy(h->d_m0, m0h.data(), m0h.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_bad(e, "copy m0");
    if ((e = cudaMalloc(&h->d_s0, (size_t)h->F * 4)) != cudaSuccess) return cuda_bad(e, "alloc s0");
    if ((e = launch_make_s(nullptr, h->d_m0, h->d_s0, h->nz, h->ny, h->nx, h->pad, h->P, h->F, h->Nz, h->Ny, h->Nx,
                           (float)(dt * dt), 0)) != cudaSuccess)
        return cuda_bad(e, "make s0");
    if ((e = cudaMalloc(&h->d_wavelet, (size_t)nt * 4)) != cudaSuccess) return cuda_bad(e, "alloc wavelet");
    if ((e = cudaMemcpy(h->d_wavelet, wh.data(), (size_t)nt * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_bad(e, "copy wavelet");
    if ((e = cudaMalloc(&h->d_src, h->src_pad.size() * 4)) != cudaSuccess) return cuda_bad(e, "alloc src");
    if ((e = cudaMemcpy(h->d_src, h->src_pad.data(), h->src_pad.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_bad(e, "copy src");
    if ((e = cudaMalloc(&h->d_rec, h->rec_pad.size() * 4)) != cudaSuccess) return cuda_bad(e, "alloc rec");
    if ((e = cudaMemcpy(h->d_rec, h->rec_pad.data(), h->rec_pad.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_bad(e, "copy rec");
    if ((e = cudaMalloc(&h->d_err, sizeof(int))) != cudaSuccess) return cuda_bad(e, "alloc err");
    if ((e = cudaMemset(h->d_err, 0, sizeof(int))) != cudaSuccess) return cuda_bad(e, "clear err");
    if (build_rec_tiles(h) != PROBE_OK) {
        std::string m = h->err;
        probe_destroy(h);
        return fail(nullptr, PROBE_ERR_CUDA, m);
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_bad(e, "create sync");
    reset_stats(h);
    *out = h;
    return PROBE_OK;
}

extern "C" void probe_destroy(probe_t h) {
    if (!h) return;
    clear_graphs(h);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    if (h->gev_in) cudaEventDestroy(h->gev_in);
    if (h->gev_out) cudaEventDestroy(h->gev_out);
    if (h->ostream) cudaStreamDestroy(h->ostream);
    for (int i = 0; i < 2; ++i) {
        if (h->ov_inc[i]) cudaEventDestroy(h->ov_inc[i]);
        if (h->ov_born[i]) cudaEventDestroy(h->ov_born[i]);
    }
    fit_cache_destroy(h);
    free_ws(h->ws);
    void* ptrs[] = {h->d_m0, h->d_s0, h->d_wavelet, h->d_src, h->d_rec, h->d_rec_tile_ptr, h->d_rec_tile_idx,
                    h->d_wrec_ptr[1], h->d_wrec_idx[1], h->d_wrec_ptr[2], h->d_wrec_idx[2],
                    h->d_rrow, h->d_uc_ptr, h->d_uc_rec, h->d_uc_pos,
                    h->d_err, h->stage_in.p, h->stage_out.p};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    delete h;
}

extern "C" const char* probe_last_error(probe_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

extern "C" const char* probe_version(void) { return "matprobe-gb300 0.1 (sm_103a)"; }

extern "C" probe_status probe_sizes(probe_t h, long long* n_model, long long* n_padded, int* ns, int* nr,
                                    int* nt) {
    if (!h) return PROBE_ERR_ARG;
    if (n_model) *n_model = h->nmodel;
    if (n_padded) *n_padded = (long long)h->Nz * h->Ny * h->Nx;
    if (ns) *ns = h->ns;
    if (nr) *nr = h->nr;
    if (nt) *nt = h->nt;
    return PROBE_OK;
}

extern "C" probe_status probe_set_option(probe_t h, int key, long long v) {
    if (!h) return PROBE_ERR_ARG;
    switch (key) {
        case PROBE_OPT_CHECK_FINITE: h->opt_check_finite = v ? 1 : 0; return PROBE_OK;
        case PROBE_OPT_SHOT_WAVE:
            if (v < 0) return fail(h, PROBE_ERR_ARG, "shot wave must be >= 0");
            h->opt_shot_wave = (int)v;
            return PROBE_OK;
        case PROBE_OPT_SHOT_GROUP:
            if (v < 0) return fail(h, PROBE_ERR_ARG, "shot group must be >= 0");
            h->opt_shot_group = (int)v;
            h->user_fixed = 1;
            return PROBE_OK;
        case PROBE_OPT_AUTOTUNE:
            h->opt_autotune = v ? 1 : 0;
            return PROBE_OK;
        case PROBE_OPT_PIPELINE_ADJ:
            if (v != 0 && v != 2 && v != 3) return fail(h, PROBE_ERR_ARG, "adjoint pipeline must be 0, 2 or 3");
            h->pipe_adj = (int)v;
            h->user_fixed = 1;
            return PROBE_OK;
        case PROBE_OPT_PIPE_ROWS:
        case PROBE_OPT_PIPE_ROWS_ADJ:
            if (v != 1 && v != 2) return fail(h, PROBE_ERR_ARG, "pipelined rows per thread must be 1 or 2");
            if (key == PROBE_OPT_PIPE_ROWS) h->ws_rows = (int)v;
            h->ws_rows_adj = (int)v;
            h->user_fixed = 1;
            return PROBE_OK;
        case PROBE_OPT_USE_GRAPH: h->opt_use_graph = v ? 1 : 0; return PROBE_OK;
        case PROBE_OPT_TBLOCK:
            if (v < 0 || v > 2) return fail(h, PROBE_ERR_ARG, "tblock must be 0, 1 or 2");
            h->user_tblock = v > 0 ? 1 : 0;
            h->opt_tblock = v > 0 ? (int)v : 1;
            return PROBE_OK;
        case PROBE_OPT_OVERLAP3D:
            h->opt_overlap3d = v ? 1 : 0;
            return PROBE_OK;
        case PROBE_OPT_PLANES3D:
            if (v != 0 && v != 32 && v != 64 && v != 128)
                return fail(h, PROBE_ERR_ARG, "planes3d must be 0, 32, 64 or 128");
            h->user_zc3d = v ? 1 : 0;
            h->zc3d = v ? (int)v : kZC3D;
            return PROBE_OK;
        case PROBE_OPT_CLUSTER3D:
            if (v < 0 || v > 3) return fail(h, PROBE_ERR_ARG, "cluster3d must be 0..3");
            h->opt_cluster3d = (int)v;
            free_ws(h->ws);  // the adjoint's image and injection buffers depend on it
            return PROBE_OK;
        case PROBE_OPT_TIMING:
            if (v < 0 || v > 2) return fail(h, PROBE_ERR_ARG, "timing must be 0, 1 or 2");
            h->opt_timing = (int)v;
            return PROBE_OK;
        case PROBE_OPT_DTT_HISTORY:
            h->opt_dtt_history = v ? 1 : 0;
            free_ws(h->ws);
            return PROBE_OK;
        case PROBE_OPT_PIPELINE:
            if (v != 0 && v != 2 && v != 3) return fail(h, PROBE_ERR_ARG, "pipeline must be 0, 2 or 3");
            h->opt_pipeline = (int)v;
            h->pipe_adj = (int)v;
            h->pipe_inc = (int)v;
            h->user_fixed = 1;
            return PROBE_OK;
        case PROBE_OPT_TILE_Z:
            if (v != 0 && v != 16 && v != 32) return fail(h, PROBE_ERR_ARG, "tile_z must be 0, 16 or 32");
            h->opt_tile_z = (int)v;
            return set_tile_z(h, v ? (int)v : 16);
    }
    return fail(h, PROBE_ERR_ARG, "unknown option");
}

extern "C" probe_status probe_diag_wait_timeout(probe_t h, int timeout_ms, probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (timeout_ms < 1 || timeout_ms > 10000) return fail(h, PROBE_ERR_ARG, "timeout_ms must be in [1, 10000]");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_diag_wait(h->d_err, (unsigned long long)timeout_ms * 1000000ull, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostic wait launch");
    return check_dev_error(h, st);
}

namespace {
probe_status finish_timing(probe_t h);
}

extern "C" probe_status probe_get_stats(probe_t h, probe_stats* out) {
    if (!h || !out) return PROBE_ERR_ARG;
    TRY(finish_timing(h));
    *out = h->stats;
    return PROBE_OK;
}

// ---------------------------------------------------------------------------
// Operators
// ---------------------------------------------------------------------------
namespace {

enum Op { OP_F, OP_FADJ, OP_H, OP_NONLIN, OP_GRAD };

probe_status ensure_events(probe_t h, int n) {
    while ((int)h->events.size() < n) {
        cudaEvent_t e;
        CK(h, cudaEventCreate(&e));
        h->events.push_back(e);
    }
    return PROBE_OK;
}

double elapsed(probe_t h, int a, int b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->events[a], h->events[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return ms;
}

// Per-sweep times of the last timed call, from the events each wave recorded:
// 0-1 forward; in checkpoint mode then per segment (recompute start, adjoint start),
// in history mode 3-4 the adjoint sweep.
probe_status finish_timing(probe_t h) {
    if (!h->tp.pending) return PROBE_OK;
    h->tp.pending = 0;
    CK(h, cudaEventSynchronize(h->ev_end));
    double ms_f = 0, ms_r = 0, ms_a = 0;
    for (int wv = 0; wv < h->tp.nwaves; ++wv) {
        const int b = wv * h->tp.nev;
        ms_f += elapsed(h, b + 0, b + 1);
        if (h->tp.ckpt && h->tp.hist) {
            ms_a += elapsed(h, b + 3, b + 4);
        } else if (h->tp.ckpt) {
            int ev = 2;
            for (int k = h->nck - 1; k >= 0; --k) {
                const int k0 = k * h->K, k1 = std::min(k0 + h->K, h->nt - 1);
                if (k0 >= k1) continue;
                ms_r += elapsed(h, b + ev, b + ev + 1);
                ms_a += elapsed(h, b + ev + 1, b + ev + 2);  // adjoint: recompute end to next segment
                ev += 2;
            }
        }
    }
    h->stats.ms_forward = ms_f;
    h->stats.ms_recompute = ms_r;
    h->stats.ms_adjoint = ms_a;
    h->stats.ms_total = ms_f + ms_r + ms_a;
    return PROBE_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: time a few steps of each kernel variant on the real workspace.
// ---------------------------------------------------------------------------
probe_status time_steps(probe_t h, cudaStream_t st, float* ms, const std::function<probe_status(int)>& step,
                        int reps) {
    TRY(ensure_events(h, 2));
    TRY(step(0));  // warm-up (also configures the kernel)
    CK(h, cudaEventRecord(h->events[0], st));
    for (int i = 0; i < reps; ++i) TRY(step(i));
    CK(h, cudaEventRecord(h->events[1], st));
    CK(h, cudaEventSynchronize(h->events[1]));
    CK(h, cudaEventElapsedTime(ms, h->events[0], h->events[1]));
    return PROBE_OK;
}

// base: the jobs of the first shot wave (one per model), exactly as the sweep will
// run them (source positions uploaded, data pointers set).  Forward variants are
// timed on steps 0, 1, ... and adjoint variants on steps nt-1, nt-2, ... with the
// Dtt slot advancing as in the sweep (so the repeated launches do not find their
// inputs in L2); the sweep itself rewrites every value the trial launches write.
// The result (forward variant, adjoint variant, shots per adjoint CTA) is kept on
// h under key; *group receives the shot group (0: keep each handle's own).
probe_status autotune_2d(probe_t h, const std::vector<long long>& key, std::vector<Job> base, FwdKind kind,
                         bool adjoint, bool time_it, cudaStream_t st, int* group) {
    *group = 0;
    if (!h->opt_autotune || h->user_fixed || h->ndim != 2 || h->tile_z != kPipeTZ || h->nt < 3) return PROBE_OK;
    for (const TunedEntry& t : h->tuned)
        if (t.key == key) {
            h->opt_pipeline = t.pipe_fwd;
            h->pipe_adj = t.pipe_adj;
            h->ws_rows = t.rows;
            h->ws_rows_adj = t.rows_adj;
            if (!h->user_tblock) h->opt_tblock = t.tblock;
            *group = t.group;
            return PROBE_OK;
        }
    if (!time_it) return PROBE_OK;
    int maxW = 1;
    for (const Job& jb : base) maxW = std::max(maxW, jb.W);
    const int saved_timing = h->opt_timing;
    h->opt_timing = 0;
    auto sweep_for = [&](int shot_group, Sweep* sw) {
        sw->jobs = base;
        for (Job& jb : sw->jobs) {
            jb.shot_group = std::min(shot_group, jb.W);
            jb.groups = (jb.W + jb.shot_group - 1) / jb.shot_group;
        }
        return prepare_sweep(*sw, h, st);
    };
    probe_status rc = PROBE_OK;
    int best_fwd = h->opt_pipeline, best_adj = h->pipe_adj, best_grp = std::min(4, maxW), best_rows = h->ws_rows;
    int best_rows_adj = h->ws_rows_adj;
    // candidates are timed round-robin, three rounds, keeping each one's fastest round
    constexpr int kRounds = 3, kReps = 24;
    int best_tb = h->opt_tblock;
    {
        // candidates 0-4: one level per launch (one tile per CTA; pipelined S x R); 5: two levels per
        // launch (time-blocked, one tile per CTA), timed per level; the pipelined candidates also set
        // the adjoint's rows per thread
        const int pipes[6] = {0, 2, 3, 2, 3, 0}, rows[6] = {1, 1, 1, 2, 2, 1};
        const int ncand = (kind == FWD_BORN && !h->user_tblock && h->ws.u4 && h->nt >= 4) ? 6 : 5;
        float t[6] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
        for (int r = 0; r < kRounds && rc == PROBE_OK; ++r)
            for (int c = 0; c < ncand && rc == PROBE_OK; ++c) {
                h->opt_pipeline = pipes[c];
                h->ws_rows = rows[c];
                Sweep sw;
                float ms = 0.f;
                if ((rc = sweep_for(1, &sw)) != PROBE_OK) break;
                const bool hist = base[0].h->ws.history != 0;
                if (c == 5) {  // two levels per launch: half the launches for the same levels
                    auto fwd2 = [&](int i) {
                        const int n = (2 * i) % (h->nt - 2);
                        return launch_fwd_tb(sw, kind, n, true, hist ? n : 0);
                    };
                    if ((rc = time_steps(h, st, &ms, fwd2, kReps / 2)) != PROBE_OK) break;
                } else {
                    auto fwd = [&](int i) {
                        const int n = i % (h->nt - 1);
                        return launch_fwd_step(sw, kind, n, hist ? n : 0);
                    };
                    if ((rc = time_steps(h, st, &ms, fwd, kReps)) != PROBE_OK) break;
                }
                t[c] = std::min(t[c], ms);
            }
        if (rc == PROBE_OK) {
            const int c5 = (int)(std::min_element(t, t + 5) - t);  // best one-level variant
            best_fwd = pipes[c5];
            best_rows = rows[c5];
            if (ncand == 6) best_tb = (t[5] < t[c5]) ? 2 : 1;
        }
    }
    if (rc == PROBE_OK && adjoint) {
        struct Cand {
            int pipe, rows, grp;
        };
        std::vector<Cand> cand;
        for (int grp : {1, 2, 4, 8}) {
            if (grp > 1 && grp >= 2 * maxW) continue;
            cand.push_back({0, 1, grp});
            for (int R : {1, 2}) cand.push_back({2, R, grp});
        }
        std::vector<float> t(cand.size(), 1e30f);
        for (int r = 0; r < kRounds && rc == PROBE_OK; ++r)
            for (size_t c = 0; c < cand.size() && rc == PROBE_OK; ++c) {
                h->pipe_adj = cand[c].pipe;
                h->ws_rows_adj = cand[c].rows;
                Sweep sw;
                float ms = 0.f;
                if ((rc = sweep_for(cand[c].grp, &sw)) != PROBE_OK) break;
                auto adj = [&](int i) {
                    const int n = h->nt - 1 - i % (h->nt - 1);
                    return launch_adj_step(sw, n, (n - 1) % std::max(1, base[0].h->ws.dtt_slots));
                };
                if ((rc = time_steps(h, st, &ms, adj, kReps)) != PROBE_OK) break;
                t[c] = std::min(t[c], ms);
            }
        if (rc == PROBE_OK) {
            const Cand& bc = cand[(size_t)(std::min_element(t.begin(), t.end()) - t.begin())];
            best_adj = bc.pipe;
            best_grp = bc.grp;
            if (bc.pipe) best_rows_adj = bc.rows;
        }
    }
    h->ws_rows = best_rows;
    h->ws_rows_adj = best_rows_adj;
    h->opt_timing = saved_timing;
    h->opt_pipeline = best_fwd;
    h->pipe_adj = best_adj;
    if (!h->user_tblock) h->opt_tblock = best_tb;
    if (rc != PROBE_OK) return rc;
    *group = best_grp;
    TunedEntry t;
    t.key = key;
    t.pipe_fwd = best_fwd;
    t.pipe_adj = best_adj;
    t.group = best_grp;
    t.rows = best_rows;
    t.rows_adj = best_rows_adj;
    t.tblock = h->opt_tblock;
    h->tuned.push_back(t);
    return PROBE_OK;
}

// Run one operator on one model.  dm: device [nb][n]; data_user: device [nb][ns][nt][nr] (F / F*)
// or [ns][nt][nr] (nonlinear / gradient); img_out: device [nb][n].
probe_status run_op(probe_t h, Op op, const float* dm_dev, const float* data_in, float* data_out,
                    float* img_out, int nb, const float* s, cudaStream_t st) {
    const bool need_ckpt = (op == OP_FADJ || op == OP_H || op == OP_GRAD);
    const bool need_data = (op == OP_H);
    const int nbw = (op == OP_NONLIN || op == OP_GRAD) ? 1 : nb;
    const int W = plan_wave(h, nbw, need_ckpt, need_data);
    TRY(ensure_ws(h, W, nbw, need_ckpt, need_data));
    Workspace& w = h->ws;
    int G = 0;
    reset_stats(h);
    h->stats.shot_wave = W;
    if (op == OP_F || op == OP_H) {
        CK(h, cudaMemsetAsync(w.dm, 0, (size_t)nb * h->F * 4, st));
        cudaError_t e = launch_embed(dm_dev, w.dm, nb, h->nz, h->nx, h->ny, h->pad, h->Nz, h->Nx, h->Ny, h->P,
                                     h->F, 1.0f, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "embed dm");
    }
    const int nwaves = (h->ns + W - 1) / W;
    const int nev = 3 + 2 * h->nck + 2;
    if (h->opt_timing) {
        TRY(ensure_events(h, nwaves * nev));
        if (!h->ev_end) CK(h, cudaEventCreate(&h->ev_end));
    }
    h->tp.pending = 0;
    for (int wv = 0; wv < nwaves; ++wv) {
        const int j0 = wv * W;
        h->ev_base = wv * nev;
        const int Wv = std::min(W, h->ns - j0);
        CK(h, cudaMemcpyAsync(w.src_wave, h->src_pad.data() + (size_t)h->ndim * j0, (size_t)Wv * h->ndim * 4,
                              cudaMemcpyHostToDevice, st));
        Sweep sw;
        Job jb;
        jb.h = h;
        jb.j0 = j0;
        jb.W = Wv;
        jb.nb = nbw;
        jb.s = s;
        const long long tr = (long long)h->nt * h->nr;
        switch (op) {
            case OP_F:
                jb.data = data_out + (long long)j0 * tr;
                jb.dss = tr;
                jb.dts = (long long)h->ns * tr;
                break;
            case OP_FADJ:
                jb.rdata = data_in + (long long)j0 * tr;
                jb.dss = tr;
                jb.dts = (long long)h->ns * tr;
                break;
            case OP_H:
                jb.data = w.data;
                jb.rdata = w.data;
                jb.dss = (long long)nbw * tr;
                jb.dts = tr;
                break;
            case OP_NONLIN:
                jb.data = data_out + (long long)j0 * tr;
                jb.dss = tr;
                jb.dts = 0;
                break;
            case OP_GRAD:
                jb.rdata = data_in + (long long)j0 * tr;
                jb.dss = tr;
                jb.dts = 0;
                break;
        }
        FwdKind kind = (op == OP_F || op == OP_H) ? FWD_BORN
                       : (op == OP_NONLIN)        ? FWD_INCIDENT_SAMPLE
                                                  : FWD_INCIDENT;
        if (wv == 0) {
            if (h->ndim == 2) {
                jb.shot_group = pick_group(h, W);
                jb.groups = (Wv + jb.shot_group - 1) / jb.shot_group;
                const std::vector<long long> tkey = {(long long)kind, (long long)need_ckpt, Wv, nbw};
                int grp = 0;
                TRY(autotune_2d(h, tkey, {jb}, kind, need_ckpt, true, st, &grp));
                if (grp > 0) h->opt_shot_group = grp;
            }
            G = (W + pick_group(h, W) - 1) / pick_group(h, W);
            h->stats.shot_group = pick_group(h, W);
            const bool piped = h->ndim == 2 && h->tile_z == kPipeTZ;
            h->stats.pipeline_forward = piped ? h->opt_pipeline : 0;
            h->stats.pipeline_adjoint = piped ? h->pipe_adj : 0;
            if (h->ndim == 3) TRY(autotune_3d(jb, kind, need_ckpt, st));
            h->stats.planes_3d = (h->ndim == 3) ? h->zc3d : 0;
            if (h->ndim == 3) {  // 0 one barrier per plane, 2 producer warp, 3 refill by the last compute warp
                h->stats.pipeline_forward = !(h->opt_cluster3d & 1) ? h->opt_pipeline : 0;
                h->stats.pipeline_incident = !(h->opt_cluster3d & 1) ? h->pipe_inc : 0;
                h->stats.pipeline_adjoint = (adj3d_ws(h) && (h->nband == 0 || w.inj)) ? h->pipe_adj : 0;
            }
            h->stats.pipeline_rows = piped ? h->ws_rows : 0;
            h->stats.pipeline_rows_adjoint = piped ? h->ws_rows_adj : 0;
            h->stats.time_block = (h->ndim == 2 && h->tile_z == kPipeTZ && w.u4) ? h->opt_tblock : 1;
            if (need_ckpt) {
                CK(h, cudaMemsetAsync(w.img, 0, (size_t)G * nbw * h->F * 4, st));
                CK(h, cudaMemsetAsync(w.comp, 0, (size_t)G * nbw * h->F * 4, st));
            }
        }
        jb.shot_group = pick_group(h, W);
        jb.groups = (Wv + jb.shot_group - 1) / jb.shot_group;
        if (h->ndim == 3) {
            Count3 c3;
            record(h, 0, st);
            TRY(run_forward3d(jb, kind, need_ckpt, st, c3));
            record(h, 1, st);
            if (need_ckpt) TRY(run_adjoint3d(jb, st, c3));
            h->stats.launches_forward += c3.fwd;
            h->stats.launches_recompute += c3.rec;
            h->stats.launches_adjoint += c3.adj;
            h->stats.launches_total += c3.fwd + c3.rec + c3.adj + c3.other;
        } else {
            sw.jobs.push_back(jb);
            const std::vector<long long> key = {(long long)op, (long long)kind, (long long)need_ckpt, Wv, nbw, j0,
                                                (long long)(size_t)jb.data, (long long)(size_t)jb.rdata,
                                                (long long)(size_t)jb.s, h->ws.generation, h->opt_pipeline, h->pipe_adj, h->ws_rows, h->ws_rows_adj, h->opt_timing, h->opt_tblock,
                                                jb.shot_group, h->tile_z, h->nt};
            long long cnt[4] = {0, 0, 0, 0};
            TRY(run_maybe_graph(h, key, st, cnt, [&](cudaStream_t ss) -> probe_status {
                Sweep sw2;
                sw2.jobs = sw.jobs;
                TRY(prepare_sweep(sw2, h, ss));
                record(h, 0, ss);
                TRY(run_forward(sw2, kind, need_ckpt));
                record(h, 1, ss);
                if (need_ckpt) TRY(run_adjoint(sw2));
                cnt[0] = sw2.launches_fwd;
                cnt[1] = sw2.launches_rec;
                cnt[2] = sw2.launches_adj;
                cnt[3] = sw2.launches_other;
                return PROBE_OK;
            }));
            sw.launches_fwd = cnt[0];
            sw.launches_rec = cnt[1];
            sw.launches_adj = cnt[2];
            sw.launches_other = cnt[3];
            finish_stats(h, sw, nwaves);
        }
        const double cells = (double)h->Nz * h->Ny * h->Nx;
        const double steps = h->nt - 1;
        const int nfields = (kind == FWD_BORN) ? 1 + nbw : 1;
        h->stats.cell_updates_forward += cells * steps * Wv * nfields;
        // algorithmic bytes: incident 16 B (u^n, u^{n-1}, s, write), Born +16 B per trial
        // (du^n, du^{n-1}, dm, write); +4 B Dtt write in the recompute.  The 3D one-field kernels
        // (no cluster fusion) also write Dtt u^n (4 B) and read it and s once per trial (8 B).
        const bool hist = w.history != 0;
        const bool split3 = h->ndim == 3 && kind == FWD_BORN && !((h->opt_cluster3d & 1) && nbw + 1 <= 8);
        // 2D with two levels per launch: per cell and level (10 + 10 nb) bytes for the Born
        // forward (u^n, u^{n-1}, s, two writes, per trial likewise, every other level) and 14 bytes
        // for the recompute (with its two Dtt writes)
        const bool tb2 = h->ndim == 2 && h->opt_tblock == 2 && h->tile_z == kPipeTZ && w.u4;
        if (tb2 && kind == FWD_BORN)
            h->stats.bytes_forward += cells * steps * Wv * (10.0 + 10.0 * nbw + (hist ? 4.0 : 0.0));
        else
            h->stats.bytes_forward += cells * steps * Wv *
                                      (16.0 + (kind == FWD_BORN ? 16.0 * nbw : 0.0) + (hist ? 4.0 : 0.0) +
                                       (split3 ? 4.0 + 8.0 * nbw : 0.0));
        if (need_ckpt) {
            if (!hist) {
                h->stats.cell_updates_recompute += cells * steps * Wv;
                h->stats.bytes_recompute += cells * steps * Wv * (tb2 ? 14.0 : 20.0);
            }
            h->stats.cell_updates_adjoint += cells * steps * Wv * nbw;
            // adjoint: per (shot, trial) mu^{n+1}, mu^{n+2}, write mu^n = 12 B; per shot Dtt 4 B;
            // s 4 B and image traffic per (group, trial) amortised over the group
            // (3D one-field adjoint with Kahan: 8 B segment-image read-modify-write per step, the
            //  Kahan fold of 20 B per cell once per segment)
            const bool seg3 = w.seg != nullptr;
            const double img_b = seg3 ? 8.0 + 20.0 / h->K : (h->kahan ? 16.0 : 8.0);
            h->stats.bytes_adjoint += cells * steps * (12.0 * Wv * nbw + 4.0 * Wv +
                                                       (double)jb.groups * (4.0 + img_b * nbw));
        }
    }
    h->ev_base = 0;
    if (need_ckpt && img_out) {
        cudaError_t e = launch_extract_images(w.img, w.comp, G, (long long)nbw * h->F, nbw, h->F, img_out, h->nz,
                                              h->ny, h->nx, h->pad, h->Ny, h->P, h->kahan != 0, false, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "image extraction");
        h->stats.launches_total++;
    }
    if (h->opt_timing) {
        CK(h, cudaEventRecord(h->ev_end, st));
        h->tp.pending = 1;
        h->tp.nwaves = nwaves;
        h->tp.nev = nev;
        h->tp.ckpt = need_ckpt && h->opt_timing == 1;
        h->tp.hist = w.history;
    }
    return PROBE_OK;
}

probe_status finish_call(probe_t h, cudaStream_t st, bool sync, const float* check, long long ncheck) {
    if (h->opt_check_finite && check && ncheck > 0) {
        cudaError_t e = launch_check_finite(check, ncheck, h->d_err, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "finite check");
        sync = true;
    }
    CK(h, cudaGetLastError());
    if (sync) TRY(check_dev_error(h, st));
    return PROBE_OK;
}

}  // namespace

extern "C" probe_status probe_apply_F(probe_t h, const float* dm, float* d, int nb, probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (nb < 0) return fail(h, PROBE_ERR_ARG, "nb must be >= 0");
    if (nb == 0) return PROBE_OK;
    if (!dm || !d) return fail(h, PROBE_ERR_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    bool hin = false;
    const float* dmd = nullptr;
    TRY(stage_input(h, dm, (size_t)nb * h->nmodel, h->stage_in, &dmd, st, &hin));
    const size_t nd = (size_t)nb * h->ns * h->nt * h->nr;
    const bool hout = !is_device_ptr(d);
    float* dd = d;
    if (hout) {
        TRY(ensure_buf(h, h->stage_out, nd * 4));
        dd = (float*)h->stage_out.p;
    }
    TRY(run_op(h, OP_F, dmd, nullptr, dd, nullptr, nb, h->d_s0, st));
    TRY(finish_call(h, st, hin || hout, dd, (long long)nd));
    if (hout) {
        CK(h, cudaMemcpyAsync(d, dd, nd * 4, cudaMemcpyDeviceToHost, st));
        CK(h, cudaStreamSynchronize(st));
    }
    return PROBE_OK;
}

extern "C" probe_status probe_apply_Fadj(probe_t h, const float* d, float* img, int nb, probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (nb < 0) return fail(h, PROBE_ERR_ARG, "nb must be >= 0");
    if (nb == 0) return PROBE_OK;
    if (!d || !img) return fail(h, PROBE_ERR_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    bool hin = false;
    const float* dd = nullptr;
    const size_t nd = (size_t)nb * h->ns * h->nt * h->nr;
    TRY(stage_input(h, d, nd, h->stage_in, &dd, st, &hin));
    const bool hout = !is_device_ptr(img);
    float* io = img;
    if (hout) {
        TRY(ensure_buf(h, h->stage_out, (size_t)nb * h->nmodel * 4));
        io = (float*)h->stage_out.p;
    }
    TRY(run_op(h, OP_FADJ, nullptr, dd, nullptr, io, nb, h->d_s0, st));
    TRY(finish_call(h, st, hin || hout, io, (long long)nb * h->nmodel));
    if (hout) {
        CK(h, cudaMemcpyAsync(img, io, (size_t)nb * h->nmodel * 4, cudaMemcpyDeviceToHost, st));
        CK(h, cudaStreamSynchronize(st));
    }
    return PROBE_OK;
}

extern "C" probe_status probe_apply_H(probe_t h, const float* dm, float* Hdm, int nb, probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (nb < 0) return fail(h, PROBE_ERR_ARG, "nb must be >= 0");
    if (nb == 0) return PROBE_OK;
    if (!dm || !Hdm) return fail(h, PROBE_ERR_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    bool hin = false;
    const float* dmd = nullptr;
    TRY(stage_input(h, dm, (size_t)nb * h->nmodel, h->stage_in, &dmd, st, &hin));
    const bool hout = !is_device_ptr(Hdm);
    float* o = Hdm;
    if (hout) {
        TRY(ensure_buf(h, h->stage_out, (size_t)nb * h->nmodel * 4));
        o = (float*)h->stage_out.p;
    }
    TRY(run_op(h, OP_H, dmd, nullptr, nullptr, o, nb, h->d_s0, st));
    TRY(finish_call(h, st, hin || hout, o, (long long)nb * h->nmodel));
    if (hout) {
        CK(h, cudaMemcpyAsync(Hdm, o, (size_t)nb * h->nmodel * 4, cudaMemcpyDeviceToHost, st));
        CK(h, cudaStreamSynchronize(st));
    }
    return PROBE_OK;
}

extern "C" probe_status probe_forward_nonlinear(probe_t h, const float* m, float* d, probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (!m || !d) return fail(h, PROBE_ERR_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    bool hin = false;
    const float* md = nullptr;
    TRY(stage_input(h, m, (size_t)h->nmodel, h->stage_in, &md, st, &hin));
    const size_t nd = (size_t)h->ns * h->nt * h->nr;
    const bool hout = !is_device_ptr(d);
    float* dd = d;
    if (hout) {
        TRY(ensure_buf(h, h->stage_out, nd * 4));
        dd = (float*)h->stage_out.p;
    }
    TRY(ensure_ws(h, plan_wave(h, 1, 0, 0), 1, 0, 0));
    // positivity of m is the caller's responsibility; non-finite values are caught by the output check
    cudaError_t e = launch_make_s(md, h->d_m0, h->ws.s_tmp, h->nz, h->ny, h->nx, h->pad, h->P, h->F, h->Nz, h->Ny,
                                  h->Nx, (float)(h->dt * h->dt), st);
    if (e != cudaSuccess) return cuda_fail(h, e, "make s");
    TRY(run_op(h, OP_NONLIN, nullptr, nullptr, dd, nullptr, 1, h->ws.s_tmp, st));
    TRY(finish_call(h, st, hin || hout, dd, (long long)nd));
    if (hout) {
        CK(h, cudaMemcpyAsync(d, dd, nd * 4, cudaMemcpyDeviceToHost, st));
        CK(h, cudaStreamSynchronize(st));
    }
    return PROBE_OK;
}

extern "C" probe_status probe_gradient(probe_t h, const float* m, const float* resid, float* g,
                                       probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (!m || !resid || !g) return fail(h, PROBE_ERR_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    bool hin1 = false;
    const float* md = nullptr;
    const float* rd = nullptr;
    // stage the model in stage_out's spare room is not possible; use two buffers
    const size_t nd = (size_t)h->ns * h->nt * h->nr;
    TRY(stage_input(h, resid, nd, h->stage_in, &rd, st, &hin1));
    DevBuf mbuf;
    if (!is_device_ptr(m)) {
        TRY(ensure_buf(h, mbuf, (size_t)h->nmodel * 4));
        CK(h, cudaMemcpyAsync(mbuf.p, m, (size_t)h->nmodel * 4, cudaMemcpyHostToDevice, st));
        md = (const float*)mbuf.p;
    } else
        md = m;
    const bool hout = !is_device_ptr(g);
    float* go = g;
    DevBuf gbuf;
    if (hout) {
        TRY(ensure_buf(h, gbuf, (size_t)h->nmodel * 4));
        go = (float*)gbuf.p;
    }
    probe_status st_ = PROBE_OK;
    do {
        st_ = ensure_ws(h, plan_wave(h, 1, 1, 0), 1, 1, 0);
        if (st_ != PROBE_OK) break;
        cudaError_t e = launch_make_s(md, h->d_m0, h->ws.s_tmp, h->nz, h->ny, h->nx, h->pad, h->P, h->F, h->Nz,
                                      h->Ny, h->Nx, (float)(h->dt * h->dt), st);
        if (e != cudaSuccess) {
            st_ = cuda_fail(h, e, "make s");
            break;
        }
        st_ = run_op(h, OP_GRAD, nullptr, rd, nullptr, go, 1, h->ws.s_tmp, st);
        if (st_ != PROBE_OK) break;
        st_ = finish_call(h, st, true, go, h->nmodel);
        if (st_ != PROBE_OK) break;
        if (hout) {
            cudaError_t e2 = cudaMemcpyAsync(g, go, (size_t)h->nmodel * 4, cudaMemcpyDeviceToHost, st);
            if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
            if (e2 != cudaSuccess) st_ = cuda_fail(h, e2, "copy gradient");
        }
    } while (0);
    cudaStreamSynchronize(st);
    if (mbuf.p) cudaFree(mbuf.p);
    if (gbuf.p) cudaFree(gbuf.p);
    return st_;
}

extern "C" probe_status probe_apply_H_group(const probe_t* models, int nmodels, const float* const* dm,
                                            float* const* Hdm, const int* nb, probe_stream_t stream) {
    if (!models || nmodels < 1 || nmodels > kMaxModels || !dm || !Hdm || !nb)
        return fail(nmodels >= 1 && models ? models[0] : nullptr, PROBE_ERR_ARG, "invalid group arguments");
    probe_t h0 = models[0];
    if (!h0) return PROBE_ERR_ARG;
    if (nmodels == 1) return probe_apply_H(h0, dm[0], Hdm[0], nb[0], stream);
    for (int k = 0; k < nmodels; ++k) {
        probe_t h = models[k];
        if (!h) return fail(h0, PROBE_ERR_ARG, "NULL handle in group");
        for (int j = 0; j < k; ++j)
            if (models[j] == h) return fail(h0, PROBE_ERR_ARG, "a handle appears twice in the group");
        if (nb[k] < 1) return fail(h0, PROBE_ERR_ARG, "every model of a group needs nb >= 1");
        if (!dm[k] || !Hdm[k]) return fail(h0, PROBE_ERR_ARG, "NULL array in group");
        if (h->ndim != 2) return fail(h0, PROBE_ERR_ARG, "group launches handle 2D grids");
        if (h->nt != h0->nt || h->K != h0->K || std::fabs(h->dt - h0->dt) > 1e-12 * h0->dt)
            return fail(h0, PROBE_ERR_ARG, "group models must share nt, dt and the checkpoint stride");
        if (h->tile_z != h0->tile_z || h->kahan != h0->kahan)
            return fail(h0, PROBE_ERR_ARG, "group models must share the tile height and the Kahan option");
    }
    cudaStream_t st = (cudaStream_t)stream;
    Sweep sw;
    std::vector<float*> outs(nmodels);
    std::vector<bool> host_out(nmodels);
    bool any_host = false;
    reset_stats(h0);
    h0->tp.pending = 0;  // this call's times are formed below
    for (int k = 0; k < nmodels; ++k) {
        probe_t h = models[k];
        bool hin = false;
        const float* dmd = nullptr;
        TRY(stage_input(h, dm[k], (size_t)nb[k] * h->nmodel, h->stage_in, &dmd, st, &hin));
        host_out[k] = !is_device_ptr(Hdm[k]);
        outs[k] = Hdm[k];
        if (host_out[k]) {
            TRY(ensure_buf(h, h->stage_out, (size_t)nb[k] * h->nmodel * 4));
            outs[k] = (float*)h->stage_out.p;
        }
        any_host = any_host || hin || host_out[k];
        TRY(ensure_ws(h, h->ns, nb[k], 1, 1));  // every shot of every model resident
        Workspace& w = h->ws;
        CK(h, cudaMemsetAsync(w.dm, 0, (size_t)nb[k] * h->F * 4, st));
        cudaError_t e = launch_embed(dmd, w.dm, nb[k], h->nz, h->nx, 1, h->pad, h->Nz, h->Nx, 1, h->P, h->F, 1.0f, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "embed dm");
        CK(h, cudaMemcpyAsync(w.src_wave, h->src_pad.data(), (size_t)h->ns * 2 * 4, cudaMemcpyHostToDevice, st));
        Job jb;
        jb.h = h;
        jb.j0 = 0;
        jb.W = h->ns;
        jb.nb = nb[k];
        jb.s = h->d_s0;
        jb.shot_group = pick_group(h, h->ns);
        jb.groups = (jb.W + jb.shot_group - 1) / jb.shot_group;
        const long long tr = (long long)h->nt * h->nr;
        jb.data = w.data;
        jb.rdata = w.data;
        jb.dss = (long long)nb[k] * tr;
        jb.dts = tr;
        sw.jobs.push_back(jb);
    }
    // kernel variants and shot group for this group of workloads (the result is kept on h0)
    std::vector<long long> key = {-1, (long long)FWD_BORN, 1, nmodels};
    for (const Job& jb : sw.jobs) {
        key.push_back((long long)(size_t)jb.h);
        key.push_back(jb.W);
        key.push_back(jb.nb);
    }
    int grp = 0;
    TRY(autotune_2d(h0, key, sw.jobs, FWD_BORN, true, true, st, &grp));
    for (Job& jb : sw.jobs) {
        if (grp > 0) jb.shot_group = std::min(grp, jb.W);
        jb.groups = (jb.W + jb.shot_group - 1) / jb.shot_group;
        Workspace& w = jb.h->ws;
        CK(jb.h, cudaMemsetAsync(w.img, 0, (size_t)jb.groups * jb.nb * jb.h->F * 4, st));
        CK(jb.h, cudaMemsetAsync(w.comp, 0, (size_t)jb.groups * jb.nb * jb.h->F * 4, st));
    }
    h0->stats.shot_group = sw.jobs[0].shot_group;
    h0->stats.pipeline_forward = h0->tile_z == kPipeTZ ? h0->opt_pipeline : 0;
    h0->stats.pipeline_adjoint = h0->tile_z == kPipeTZ ? h0->pipe_adj : 0;
    h0->stats.pipeline_rows = h0->tile_z == kPipeTZ ? h0->ws_rows : 0;
    h0->stats.pipeline_rows_adjoint = h0->tile_z == kPipeTZ ? h0->ws_rows_adj : 0;
    if (h0->opt_timing) TRY(ensure_events(h0, 3 + 2 * h0->nck + 2));
    // the whole group's sweeps as one graph (cached on h0 by handles, workspaces and variants)
    std::vector<long long> gkey = key;
    for (const Job& jb : sw.jobs) {
        gkey.push_back(jb.h->ws.generation);
        gkey.push_back(jb.shot_group);
    }
    gkey.push_back(h0->opt_pipeline);
    gkey.push_back(h0->pipe_adj);
    gkey.push_back(h0->ws_rows);
    gkey.push_back(h0->ws_rows_adj);
    gkey.push_back(h0->opt_timing);
    gkey.push_back(h0->tile_z);
    long long cnt[4] = {0, 0, 0, 0};
    TRY(run_maybe_graph(h0, gkey, st, cnt, [&](cudaStream_t ss) -> probe_status {
        Sweep sw2;
        sw2.jobs = sw.jobs;
        TRY(prepare_sweep(sw2, h0, ss));
        record(h0, 0, ss);
        TRY(run_forward(sw2, FWD_BORN, true));
        record(h0, 1, ss);
        TRY(run_adjoint(sw2));
        cnt[0] = sw2.launches_fwd;
        cnt[1] = sw2.launches_rec;
        cnt[2] = sw2.launches_adj;
        cnt[3] = sw2.launches_other;
        return PROBE_OK;
    }));
    sw.launches_fwd = cnt[0];
    sw.launches_rec = cnt[1];
    sw.launches_adj = cnt[2];
    sw.launches_other = cnt[3];
    finish_stats(h0, sw, 1);
    for (int k = 0; k < nmodels; ++k) {
        probe_t h = models[k];
        Workspace& w = h->ws;
        const int groups_k = sw.jobs[k].groups;
        cudaError_t e = launch_extract_images(w.img, w.comp, groups_k, (long long)nb[k] * h->F, nb[k], h->F, outs[k],
                                              h->nz, 1, h->nx, h->pad, 1, h->P, h->kahan != 0, false, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "image extraction");
        const double cells = (double)h->Nz * h->Nx, steps = h->nt - 1;
        h0->stats.cell_updates_forward += cells * steps * h->ns * (1 + nb[k]);
        h0->stats.cell_updates_recompute += cells * steps * h->ns;
        h0->stats.cell_updates_adjoint += cells * steps * h->ns * nb[k];
        // algorithmic bytes, as for probe_apply_H
        h0->stats.bytes_forward += cells * steps * h->ns * (16.0 + 16.0 * nb[k]);
        h0->stats.bytes_recompute += cells * steps * h->ns * 20.0;
        h0->stats.bytes_adjoint += cells * steps * (12.0 * h->ns * nb[k] + 4.0 * h->ns +
                                                    (double)sw.jobs[k].groups * (4.0 + (h->kahan ? 16.0 : 8.0) * nb[k]));
        TRY(finish_call(h, st, any_host, outs[k], (long long)nb[k] * h->nmodel));
    }
    if (h0->opt_timing) {
        CK(h0, cudaStreamSynchronize(st));
        h0->stats.ms_forward = elapsed(h0, 0, 1);
        int ev = 2;
        for (int kk = h0->nck - 1; kk >= 0; --kk) {
            const int k0 = kk * h0->K, k1 = std::min(k0 + h0->K, h0->nt - 1);
            if (k0 >= k1) continue;
            h0->stats.ms_recompute += elapsed(h0, ev, ev + 1);
            h0->stats.ms_adjoint += elapsed(h0, ev + 1, ev + 2);
            ev += 2;
        }
        h0->stats.ms_total = h0->stats.ms_forward + h0->stats.ms_recompute + h0->stats.ms_adjoint;
    }
    for (int k = 0; k < nmodels; ++k) {
        if (!host_out[k]) continue;
        probe_t h = models[k];
        CK(h, cudaMemcpyAsync(Hdm[k], outs[k], (size_t)nb[k] * h->nmodel * 4, cudaMemcpyDeviceToHost, st));
    }
    if (any_host) CK(h0, cudaStreamSynchronize(st));
    return PROBE_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free Born forward (probe_apply_F_noalloc).
//
// For callers that must not allocate device memory while they run -- code
// inside a region that owns a fixed, pre-reserved memory budget (an inference
// or imaging service that hands all remaining memory to its own pool), hosts
// whose framework forbids cudaMalloc/cudaFree between its own allocation
// points because they synchronise the device, or real-time loops that cannot
// afford allocation latency.  Such a caller creates the handle once at set-up
// time and then calls this entry point, which needs no memory beyond the
// caller's input and output arrays and the file-scope scratch array below.
//
// The scratch is a static __device__ array of kNoAllocScratchBytes (32 MiB);
// every GPU on which the library is loaded holds it until the process exits.
// Host code may not use the array's name as a device address, so the first
// call on each device looks its address up with cudaGetSymbolAddress (with
// that device current) and caches it; make that first call before any stream
// capture.  All calls share the array and it keeps the last call's contents:
// the state planes are cleared at the start of every wave.  Two calls whose
// work overlaps on the GPU (different streams, or different handles on the
// same device) race on the scratch and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

probe_status noalloc_scratch(probe_t h, void** out) {
    int devid = 0;
    CK(h, cudaGetDevice(&devid));
    if (devid < 0 || devid >= kNoAllocMaxDevices)
        return fail(h, PROBE_ERR_ARG, "device ordinal beyond the allocation-free path's table");
    if (!g_noalloc_addr[devid]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(h, e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[devid] = p;
    }
    *out = g_noalloc_addr[devid];
    return PROBE_OK;
}

}  // namespace

extern "C" probe_status probe_apply_F_noalloc(probe_t h, const float* dm, float* d, int nb,
                                              probe_stream_t stream) {
    if (!h) return PROBE_ERR_ARG;
    if (nb < 0) return fail(h, PROBE_ERR_ARG, "nb must be >= 0");
    if (nb == 0) return PROBE_OK;
    if (!dm || !d) return fail(h, PROBE_ERR_ARG, "NULL array");
    if (h->ndim != 2) return fail(h, PROBE_ERR_ARG, "the allocation-free path handles 2D grids");
    // per resident shot: incident (2 planes) + nb Born fields (2 planes each); plus nb dm planes
    const size_t plane = (size_t)h->F * 4;
    const size_t fixed = (size_t)nb * plane;
    const size_t per_shot = (size_t)(2 + 2 * nb) * plane;
    if (fixed + per_shot > kNoAllocScratchBytes) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "sizes beyond the allocation-free maximum: one shot with nb=%d needs %zu bytes of "
                 "scratch, the static scratch holds %zu",
                 nb, fixed + per_shot, kNoAllocScratchBytes);
        return fail(h, PROBE_ERR_ARG, buf);
    }
    if (!is_device_ptr(dm) || !is_device_ptr(d))
        return fail(h, PROBE_ERR_ARG, "the allocation-free path needs device arrays");
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    TRY(noalloc_scratch(h, &base));
    const int W = (int)std::min<size_t>((size_t)h->ns, (kNoAllocScratchBytes - fixed) / per_shot);
    float* s_dm = (float*)base;
    float* s_u = s_dm + (size_t)nb * h->F;
    float* s_f = s_u + (size_t)W * 2 * h->F;
    CUtensorMap tm_u, tm_f;
    TRY(encode_planes(h, &tm_u, s_u, W * 2, h->tile_z));
    TRY(encode_planes(h, &tm_f, s_f, W * nb * 2, h->tile_z));

    CK(h, cudaMemsetAsync(s_dm, 0, (size_t)nb * plane, st));
    cudaError_t e = launch_embed(dm, s_dm, nb, h->nz, h->nx, 1, h->pad, h->Nz, h->Nx, 1, h->P, h->F, 1.0f, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "embed dm");

    const long long tr = (long long)h->nt * h->nr;
    StepParams2D p;
    memset(&p, 0, sizeof(p));
    p.nmodels = 1;
    p.nt = h->nt;
    p.err = h->d_err;
    ModelStep2D& m = p.m[0];
    m.tm_u = tm_u;
    m.tm_f = tm_f;
    m.Nz = h->Nz;
    m.Nx = h->Nx;
    m.P = h->P;
    m.pad = h->pad;
    m.nz = h->nz;
    m.nx = h->nx;
    m.tiles_x = h->tiles_x;
    m.tiles_z = h->tiles_z;
    m.ntiles = h->ntiles;
    m.block_begin = 0;
    m.nb = nb;
    m.shot_group = 1;
    m.ngroups = 1;
    m.nbc_chunks = 1;
    m.nr = h->nr;
    m.cz = h->cz;
    m.cx = h->cx;
    const double wk[4] = {PROBE_W1, PROBE_W2, PROBE_W3, PROBE_W4};
    m.c0 = (float)(PROBE_W0 / (h->hz * h->hz) + PROBE_W0 / (h->hx * h->hx));
    for (int k = 0; k < 4; ++k) {
        m.lz[k] = (float)(wk[k] / (h->hz * h->hz));
        m.lx[k] = (float)(wk[k] / (h->hx * h->hx));
    }
    for (int mm = 0; mm < 4; ++mm) {
        double cm = 0.0;
        for (int k = mm; k < 4; ++k) cm += wk[k];
        m.cxm[mm] = (float)(cm / (h->hx * h->hx));
        m.czm[mm] = (float)(cm / (h->hz * h->hz));
    }
    m.inv_dt2 = (float)(1.0 / (h->dt * h->dt));
    m.vol_inv = (float)(1.0 / (h->hz * h->hx));
    m.F = h->F;
    m.u = s_u;
    m.f = s_f;
    m.s = h->d_s0;
    m.dm = s_dm;
    m.wavelet = h->d_wavelet;
    m.rec_tile_ptr = h->d_rec_tile_ptr;
    m.rec_tile_idx = h->d_rec_tile_idx;
    m.rec_zx = h->d_rec;
    m.data_shot_stride = tr;
    m.data_trial_stride = (long long)h->ns * tr;

    for (int j0 = 0; j0 < h->ns; j0 += W) {
        const int Wv = std::min(W, h->ns - j0);
        CK(h, cudaMemsetAsync(s_u, 0, (size_t)Wv * 2 * plane, st));
        CK(h, cudaMemsetAsync(s_f, 0, (size_t)Wv * nb * 2 * plane, st));
        m.nshots = Wv;
        m.src_zx = h->d_src + 2 * j0;
        m.data = d + (long long)j0 * tr;
        for (int n = 0; n < h->nt - 1; ++n) {
            p.n = n;
            e = launch_fwd2d(FWD_BORN, h->tile_z, p, Wv, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "forward step launch");
        }
        e = launch_sample(s_f, (long long)nb * 2 * h->F, 2 * h->F, (h->nt - 1) & 1, h->F, Wv, nb, h->d_rec, h->nr,
                          h->P, 2, 1, m.data, tr, (long long)h->ns * tr, h->nt - 1, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "receiver sampling");
    }
    return finish_call(h, st, false, d, (long long)nb * h->ns * tr);
}
