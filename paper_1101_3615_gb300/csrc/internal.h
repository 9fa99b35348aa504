// Internal (not ABI) declarations of the matrix-probing library: kernel
// parameter blocks, the per-model device state and the launcher entry points
// that the C ABI layer (probe_api.cu) drives.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/probe.h"

namespace probe {

constexpr int kMaxModels = 4;
constexpr int kTX = 64;        // 2D tile width (x), 16 float4 lanes
constexpr int kThreads = 256;  // threads per stencil CTA
constexpr int kMaxNbc = 8;     // trials per adjoint CTA (register accumulators)
constexpr int kTY3D = 16;      // 3D tile height (y)
constexpr int kZC3D = 64;      // 3D planes marched by one CTA (default; the autotuner may pick 32 or 128)
constexpr int kZCMax3D = 128;  // most 3D planes one CTA may march (size of the per-plane tables)

// ---------------------------------------------------------------------------
// Kernel parameter block of one model inside a (possibly multi-model) launch.
// Passed by value as a __grid_constant__ so the TMA descriptors live in param
// space.
// ---------------------------------------------------------------------------
struct alignas(128) ModelStep2D {
    CUtensorMap tm_u;    // incident-field planes  [W*2][Nz][P], halo box (64+8) x (TZ+8)
    CUtensorMap tm_f;    // Born / adjoint planes  [W*nb*2][Nz][P], halo box
    // pipelined kernels, tile 64 x 16R (R = ws_rows): halo boxes (64+8) x (16R+8) and plain boxes
    CUtensorMap tm_wu;
    CUtensorMap tm_wf;
    CUtensorMap tm_up;   // incident planes, plain box
    CUtensorMap tm_fp;   // Born / adjoint planes, plain box
    CUtensorMap tm_sp;   // s, one plane, plain box
    CUtensorMap tm_dmp;  // dm, nb planes, plain box
    CUtensorMap tm_dtp;  // Dtt segment buffer, W * dtt_slots planes, plain box
    CUtensorMap tm_img;  // images [groups][nb] planes, plain box (pipelined adjoint)
    CUtensorMap tm_cmp;  // their Kahan compensation
    // two-step (time-blocked) forward kernels over the four-level states u4 / f4: boxes of the tile
    // plus an 8-cell halo (80 x 32) and of the first step's region, tile plus 4 (72 x 24)
    CUtensorMap tm_u4h, tm_u4e, tm_f4h, tm_f4e;
    CUtensorMap tm_se;   // s, 72 x 24 box
    CUtensorMap tm_dme;  // dm, 72 x 24 box
    int Nz, Nx, P, pad, nz, nx;
    int tiles_x, tiles_z, ntiles;
    int ws_rows;                 // pipelined kernels: rows per thread R (tile height 16R)
    int ws_tiles_z, ws_ntiles;   // their tile grid
    const int* ws_rec_ptr;       // receivers by pipelined tile (CSR over ws_ntiles)
    const int* ws_rec_idx;
    // adjoint injection R^T r^n, prebuilt per checkpoint segment: rows that hold receivers
    // ("bands") of each (slot, shot, trial), nband x P floats per block
    const int* rrow;             // [Nz] band of a grid row, -1 without receivers
    const float* inj;            // [slots][nshots][nb][nband][P]
    int inj_slot;                // slot of this step
    int nband;
    int block_begin;   // first grid.z index of this model in the launch
    int item_begin;    // pipelined kernels: first work item of this model
    int dtt_slots;     // Dtt planes per shot in the segment buffer
    int dtt_store;     // forward Born step also writes Dtt u^n to slot dtt_slot (history mode)
    int chunk;         // adjoint: trial chunk of this launch
    int nshots;        // shots resident in this launch
    int nb;            // trials (Born / adjoint fields per shot)
    int shot_group;    // adjoint: shots handled by one CTA
    int ngroups;       // adjoint: ceil(nshots / shot_group)
    int nbc_chunks;    // adjoint: ceil(nb / NBC)
    int nr;
    int dtt_slot;      // segment-buffer slot of this step
    float cz, cx;      // sponge: eta dt/2 = cz rho_z^2 + cx rho_x^2
    float c0;          // w0 (1/hz^2 + 1/hx^2)
    float lz[4], lx[4];  // w_k / h^2 per axis, k = 1..4
    float cxm[4];        // x taps in first-difference form: sum_{k>m} w_k / hx^2, m = 0..3
    float czm[4];        // z taps in the same form (pipelined kernels): sum_{k>m} w_k / hz^2
    float inv_dt2;
    float vol_inv;     // 1 / (hz hx)
    long long F;       // floats per plane (Nz * P)
    float* u;          // incident state base
    float* f;          // Born/adjoint state base
    float* u4;         // time-blocked forward: incident levels [W][4][F], level n in plane n & 3
    float* f4;         // and Born levels [W][nb][4][F]
    const float* s;    // dt^2 / m on the padded grid [F]
    const float* dm;   // [nb][F] model perturbations (zero in the pad)
    float* dtt;        // segment buffer, Dtt u^n  [W][K][F]
    long long dtt_shot_stride;
    const float* wavelet;   // [nt]
    const int* src_zx;      // [W][2] padded source cell of each resident shot
    const int* rec_tile_ptr;  // [ntiles + 1]
    const int* rec_tile_idx;  // receivers sorted by tile
    const int* rec_zx;        // [nr][2] padded receiver cells
    float* data;              // forward output traces
    const float* rdata;       // adjoint input traces
    long long data_shot_stride, data_trial_stride;  // floats; time stride = nr
    float* img;               // [ngroups][nb][F]
    float* comp;              // Kahan compensation, same layout
    long long img_group_stride;
};

struct StepParams2D {
    int nmodels;
    int total_items;  // pipelined kernels: work items over all models
    int n;    // time index of the step (forward: u^n -> u^{n+1}; adjoint: computes mu^n)
    int two;  // time-blocked forward kernel: 1 = advance n -> n + 2, 0 = one step
    int nt;
    int* err; // device error word
    ModelStep2D m[kMaxModels];
};

// ---------------------------------------------------------------------------
// 3D: one field kind per launch; grid = (tiles_x * tiles_y * zchunks, nshots * nfield).
// ---------------------------------------------------------------------------
enum Step3Mode { STEP3_INC = 0, STEP3_INC_SAMPLE = 1, STEP3_BORN = 2, STEP3_ADJ = 3 };

struct alignas(128) ModelStep3D {
    CUtensorMap tm;    // 4D map (x, y, z, volume) over the state being differentiated
    int Nz, Ny, Nx, P, pad, nz, ny, nx;
    int tiles_x, tiles_y, zchunks, ZC;
    int nshots, nfield;  // fields per shot in this launch (1 incident, nb Born / adjoint)
    int nvol_shot;       // volumes per shot in the state buffer (2 * nfield)
    int nr;
    float cz, cy, cx;
    float lz[4], ly[4], lx[4];
    float cxm[4];        // x taps in first-difference form, sum_{k>m} w_k / hx^2
    float inv_dt2, vol_inv;
    long long F;         // floats per volume (Nz * Ny * P)
    float* state;
    const float* s;
    const float* dm;           // Born: [nb][F]
    const float* Din;          // Born: Dtt u^n of each shot; adjoint: Dtt u^{n-1}
    long long Din_shot_stride;
    float* Dout;               // incident: where Dtt u^n goes (may be null)
    long long Dout_shot_stride;
    const float* wavelet;
    const int* src;            // [W][3] padded (z, y, x)
    const int* rec_ptr;        // CSR over (tile_y * tiles_x + tile_x) * Nz + z
    const int* rec_idx;
    const int* rec_zyx;        // [nr][3] padded
    float* data;
    const float* rdata;
    long long dss, dts;
    float* img;                // adjoint: [W][nb][F] (one-field kernels) or [W / G][nb][F] (shot clusters)
    float* comp;
    int seg_first;             // one-field adjoint into a segment image: first step of the segment (img = t)
    // shot-cluster adjoint: receiver injection R^T r^n prebuilt per checkpoint segment for the
    // planes that hold receivers ("bands"), inj[slot][shot][trial][band][Ny][P], slot = n_hi - n
    const int* rrow;           // [Nz] band of a plane, -1 without receivers
    const float* inj;
    int inj_slot;
    long long inj_block;       // floats per (slot, shot, trial) block = nband * Ny * P
};

struct StepParams3D {
    int n, nt;
    int* err;
    ModelStep3D m;
    ModelStep3D m2;  // cluster kernels: the Born fields of the fused forward step
};

// pipeline: 0 one barrier per plane; 2 producer warp; 3 the last compute warp out of a slot refills it
cudaError_t launch_step3d(int mode, bool kahan, int pipeline, const StepParams3D& p, cudaStream_t st);
size_t step3d_smem_bytes();
// Fused incident + Born step on clusters of 1 + nb CTAs (m: incident, m2: Born, nb = m2.nfield <= 7).
cudaError_t launch_fwd3d_cluster(const StepParams3D& p, cudaStream_t st);
size_t fwd3d_cluster_smem_bytes();
// Adjoint + imaging on clusters of G shots (G = 1, 2, 4, 8; m.nshots % G == 0): one image per
// (shot group, trial), img [nshots / G][nb][F].
cudaError_t launch_adj3d_cluster(int G, bool kahan, const StepParams3D& p, cudaStream_t st);

// Launchers (stencil2d.cu).  `zblocks` = grid.z extent: shots (forward) or shot
// groups (adjoint) summed over the models of the launch.
enum FwdKind { FWD_INCIDENT = 0, FWD_INCIDENT_DTT = 1, FWD_BORN = 2, FWD_INCIDENT_SAMPLE = 3 };
cudaError_t launch_fwd2d(FwdKind kind, int tile_z, const StepParams2D& p, int blocks,
                         cudaStream_t st);
cudaError_t launch_adj2d(int tile_z, int nbc, bool kahan, const StepParams2D& p, int blocks,
                         int chunks, cudaStream_t st);
size_t fwd2d_smem_bytes(FwdKind kind, int tile_z);
// Time-blocked forward (two levels per launch, one 64 x 16 tile per CTA) over u4 / f4: kind
// FWD_BORN or FWD_INCIDENT_DTT; p.two selects two steps (n -> n + 2) or one.
cudaError_t launch_fwd2d_tb(FwdKind kind, const StepParams2D& p, int blocks, cudaStream_t st);
// Pipelined persistent variants (stencil2d_pipe.cu): tiles of 64 x 16R (R = m[].ws_rows, 1 or 2),
// `stages`-deep TMA ring.  They need the handle's plain tile height kPipeTZ for its receiver lists.
constexpr int kPipeTZ = 16;
cudaError_t launch_fwd2d_pipe(FwdKind kind, int stages, const StepParams2D& p, cudaStream_t st);
cudaError_t launch_adj2d_pipe(int nbc, bool kahan, int stages, const StepParams2D& p, int chunks, cudaStream_t st);
size_t pipe_smem_bytes(int stages, bool adjoint, int rows);
size_t adj2d_smem_bytes(int tile_z);
cudaError_t stencil2d_configure();  // opt-in shared memory sizes

// Auxiliary kernels (aux.cu).
cudaError_t launch_embed(const float* src_int, float* dst_pad, int nb, int nz, int nx, int ny,
                         int pad, int Nz, int Nx, int Ny, int P, long long F, float scale,
                         cudaStream_t st);
cudaError_t launch_make_s(const float* m_int, const float* m0_int, float* s_pad, int nz, int ny,
                          int nx, int pad, int P, long long F, int Nz, int Ny, int Nx, float dt2,
                          cudaStream_t st);
cudaError_t launch_extract_images(const float* img, const float* comp, int ngroups,
                                  long long group_stride, int nb, long long F, float* out,
                                  int nz, int ny, int nx, int pad, int Ny, int P, bool kahan,
                                  bool accumulate, cudaStream_t st);
cudaError_t launch_sample(const float* field, long long plane_stride_shot,
                          long long plane_stride_trial, int plane, long long F, int nshots,
                          int nb, const int* rec_zx, int nr, int P, int ndim, int Ny, float* data,
                          long long data_shot_stride, long long data_trial_stride, int n,
                          cudaStream_t st);
cudaError_t launch_check_finite(const float* a, long long n, int* err, cudaStream_t st);
cudaError_t launch_build_injection(const float* rdata, long long dss, long long dts, int nr, int n_hi, int nsteps,
                                   int nshots, int nb, int nuc, const int* uc_ptr, const int* uc_rec,
                                   const int* uc_pos, float* inj, long long block, cudaStream_t st);
// Checkpoint storage of one shot (FP32: 2 planes; FP16: 2 half planes; BF16: 3 bf16 planes).
size_t ckpt_bytes_per_shot(int dtype, long long F);
// State planes of shot j: pps planes per shot, u^n in plane pps j + p_un, u^{n-1} in pps j + p_prev
// (the two-level states: pps = 2, p_un = n & 1; the four-level states of the time-blocked forward:
// pps = 4, p_un = n & 3).  nplanes = 2 x shots.
cudaError_t launch_encode_ckpt(const float* state, int nplanes, long long F, int pps, int p_un, int p_prev, void* dst,
                               float* scales, int dtype, float* absmax_scratch, cudaStream_t st);
cudaError_t launch_decode_ckpt(const void* src, const float* scales, int nplanes, long long F, int pps, int p_un,
                               int p_prev, int dtype, float* state, cudaStream_t st);
cudaError_t launch_scale_copy(const float* src, float* dst, long long n, float a, cudaStream_t st);
// img, comp (+)= seg with Kahan compensation (n floats): the end of a checkpoint segment of the 3D
// adjoint, whose steps summed their imaging terms into the plain FP32 segment image seg.
cudaError_t launch_kahan_fold(float* img, float* comp, const float* seg, long long n, cudaStream_t st);
cudaError_t launch_diag_wait(int* err, unsigned long long limit_ns, cudaStream_t st);

}  // namespace probe
