// Definition of the library handle (struct probe_s) and the host helpers that
// the C ABI translation units share.  Internal, not part of the ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"

namespace probe {

struct WsMaps {
    CUtensorMap wu, wf;                      // halo boxes (64 + 8) x (16 rows + 8): incident, Born/adjoint
    CUtensorMap up, fp, dmp, dtp, img, cmp;  // plain 64 x 16 rows boxes
    int rows = 0;                            // R (0: not encoded)
};

struct Workspace {
    // sizing key
    int W = 0, nb = 0, with_ckpt = 0, with_data = 0, groups = 0;
    int history = 0;          // Dtt u^n kept for every step (no checkpoints)
    int dtt_slots = 0;        // Dtt planes per shot
    size_t bytes = 0;
    float* u = nullptr;       // [W][2][F]
    float* f = nullptr;       // [W][nb][2][F]
    float* u4 = nullptr;      // 2D time-blocked forward: [W][4][F] (level n in plane n & 3)
    float* f4 = nullptr;      // [W][nb][4][F]
    CUtensorMap tm_u4h, tm_u4e, tm_f4h, tm_f4e, tm_dme;  // their boxes (80 x 32, 72 x 24) and dm's
    float* dm = nullptr;      // [nb][F]
    float* data = nullptr;    // [W][nb][nt][nr]
    void* ckpt = nullptr;     // [nck][W][2][F] (fp32 or 16-bit)
    float* scales = nullptr;  // [nck][W*2]
    float* absmax = nullptr;  // [W*2]
    float* dtt = nullptr;     // [W][K][F]
    float* img = nullptr;     // [groups][nb][F]
    float* seg = nullptr;     // 3D one-field adjoint with Kahan: plain FP32 image of one checkpoint segment
    float* comp = nullptr;
    float* s_tmp = nullptr;   // [F]
    int* src_wave = nullptr;  // [W][2] padded sources of the wave
    float* inj = nullptr;     // [K][W][nb][nband][P] adjoint injection of one segment (2D)
    CUtensorMap tm_u, tm_f;
    // pipelined kernels: halo and plain boxes for tiles of 64 x 16 rows, one set for the
    // forward kernels and one for the adjoint (their row counts are chosen separately)
    WsMaps mf, ma;
    int tm_tile_z = 0;
    long long generation = 0;
};

// A captured sweep (forward + adjoint of one wave) and the key it was captured for.
struct TunedEntry {
    std::vector<long long> key;  // kind, adjoint, then shots and trials of each model (and handles for groups)
    int pipe_fwd = 2, pipe_adj = 2, group = 4, rows = 2, rows_adj = 1, tblock = 1;
};

// 3D autotuner result: refill scheme of the pipelined forward and adjoint kernels, planes per CTA.
struct Tuned3 {
    std::vector<long long> key;  // kind, adjoint, shots, trials
    int fam_fwd = 2, fam_inc = 2, fam_adj = 2, zc = 64;
};

struct GraphEntry {
    std::vector<long long> key;
    cudaGraphExec_t exec = nullptr;
    long long counts[4] = {0, 0, 0, 0};  // kernel launches inside (forward, recompute, adjoint, other)
};

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

struct FitCache;

}  // namespace probe

struct probe_s {
    std::string err;
    int ndim = 2;
    int nz = 0, ny = 1, nx = 0, pad = 0;
    int Nz = 0, Ny = 1, Nx = 0, P = 0;
    long long F = 0;
    long long nmodel = 0;
    double hz = 0, hy = 0, hx = 0, dt = 0;
    int nt = 0, ns = 0, nr = 0;
    int snap = 0, kahan = 1, K = 0, nck = 0;
    double cmax = 0;
    float cz = 0, cx = 0, cy = 0;
    std::vector<int> src_pad;  // [ns][ndim] padded
    std::vector<int> rec_pad;  // [nr][ndim] padded
    float* d_m0 = nullptr;     // interior
    float* d_s0 = nullptr;     // padded
    float* d_wavelet = nullptr;
    int* d_src = nullptr;
    int* d_rec = nullptr;
    int* d_rec_tile_ptr = nullptr;
    int* d_rec_tile_idx = nullptr;
    int tile_z = 16, tiles_x = 0, tiles_y = 1, tiles_z = 0, ntiles = 0;
    // receivers by pipelined-kernel tile (64 x 16R), R = 1, 2
    int* d_wrec_ptr[3] = {nullptr, nullptr, nullptr};
    int* d_wrec_idx[3] = {nullptr, nullptr, nullptr};
    // 2D adjoint injection: grid rows holding receivers ("bands") and the receiver cells with
    // their receivers (CSR, receiver order), built once per handle
    int* d_rrow = nullptr;       // [Nz] band index or -1
    int* d_uc_ptr = nullptr;     // [nuc + 1]
    int* d_uc_rec = nullptr;     // [nr]
    int* d_uc_pos = nullptr;     // [nuc] band * P + x
    int nband = 0, nuc = 0;
    int ws_rows = 2;             // rows per thread R of the pipelined forward kernels
    int ws_rows_adj = 1;         // and of the pipelined adjoint kernels
    int* d_err = nullptr;
    probe::Workspace ws;
    probe::DevBuf stage_in, stage_out;
    // options
    int opt_check_finite = 1, opt_shot_wave = 0, opt_shot_group = 0, opt_use_graph = 0;
    int opt_timing = 0, opt_tile_z = 0, opt_pipeline = 2, opt_dtt_history = 0;
    int opt_autotune = 1;        // time the kernel variants on first use of a shape
    int opt_cluster3d = 0;       // 3D cluster kernels: bit 0 fused forward, bit 1 shot-clustered adjoint
    int opt_tblock = 1;          // 2D Born forward and recompute: time levels per launch (1 or 2)
    int user_tblock = 0;         // the caller fixed opt_tblock (else the autotuner chooses)
    int pipe_adj = 2;            // adjoint kernel variant (the forward uses opt_pipeline)
    int pipe_inc = 2;            // 3D: ring-refill scheme of the incident step (forward and recompute)
    int opt_overlap3d = 1;       // 3D Born forward: incident step n+1 concurrent with Born step n
    int zc3d = probe::kZC3D;     // 3D: z planes marched by one CTA (32, 64 or 128)
    int user_zc3d = 0;           // the caller fixed zc3d (else the autotuner chooses)
    std::vector<probe::Tuned3> tuned3;  // 3D autotuner results by workload key
    int user_fixed = 0;          // the caller chose pipeline / shot group: no autotuning
    std::vector<probe::TunedEntry> tuned;  // autotuner results by workload key
    probe_stats stats{};
    std::vector<cudaEvent_t> events;
    // PROBE_OPT_TIMING: each shot wave records its own events (base ev_base); the sums are
    // formed when the statistics are read, after the end event, so no call synchronises
    int ev_base = 0;
    cudaEvent_t ev_end = nullptr;
    struct {
        int pending = 0, nwaves = 0, nev = 0, ckpt = 0, hist = 0;
    } tp;
    probe::FitCache* fit = nullptr;  // FFT plans and buffers of probe_fit / probe_apply_precond
    // captured sweeps (PROBE_OPT_USE_GRAPH), replayed on gstream
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    // 3D forward with the incident step n+1 overlapping the Born step n: the Born steps run on
    // ostream; ov_inc[s] / ov_born[s] mark the incident / Born step that last used Dtt slot s
    cudaStream_t ostream = nullptr;
    cudaEvent_t ov_inc[2] = {nullptr, nullptr}, ov_born[2] = {nullptr, nullptr};
    std::vector<probe::GraphEntry> graphs;
    long long graph_generation = -1;
};

namespace probe {

probe_status fail(probe_t h, probe_status st, const std::string& msg);
probe_status cuda_fail(probe_t h, cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
probe_status ensure_buf(probe_t h, DevBuf& b, size_t bytes);
void fit_cache_destroy(probe_t h);

}  // namespace probe

#define PROBE_CK(h, call)                                              \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::probe::cuda_fail(h, e_, #call); \
    } while (0)

#define PROBE_TRY(call)                \
    do {                               \
        probe_status s_ = (call);      \
        if (s_ != PROBE_OK) return s_; \
    } while (0)
