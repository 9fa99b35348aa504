// Device-side helpers shared by the sm_103a kernels of the matrix-probing library:
// mbarrier + TMA (cp.async.bulk.tensor) wrappers with time-bounded waits, the
// device error word, and small vector utilities.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace probe {

// Device error word bits (OR-ed by kernels, read by the host after a sync).
enum : int { DEVERR_TIMEOUT = 1, DEVERR_NONFINITE = 2 };

// A bounded wait gives up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Plain arrival (no transaction bytes) on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Shared-memory counter increment with acquire-release semantics at CTA scope: the caller's
// earlier accesses are ordered before it, and the thread that reads the final count sees every
// other incrementer's earlier accesses.  Returns the previous value.
__device__ __forceinline__ uint32_t atom_add_acqrel_shared(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(p)), "r"(v)
                 : "memory");
    return old;
}

// Orders this thread's generic-proxy shared-memory accesses (and those it has observed) before
// its subsequent async-proxy operations (a TMA write into a slot that was just read).
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Wait for phase `parity` of `bar`; false if it did not complete within `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// ---- thread-block clusters: distributed shared memory and cluster-scope mbarriers ----
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Shared-memory address (shared::cta window) of this CTA -> the same offset in CTA `rank` of
// the cluster (shared::cluster window).
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Asynchronous store of 16 bytes into the shared memory of another CTA of the cluster; its
// arrival decrements the transaction count of that CTA's mbarrier `remote_bar` by 16 bytes, so
// the data and the signal travel together (no fence on the storing thread).
__device__ __forceinline__ void st_async4(uint32_t remote_addr, const float4& v, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     remote_addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(remote_bar)
                 : "memory");
}

// Plain (relaxed) arrival on an mbarrier of another CTA of the cluster: used to hand a buffer
// back once the values read from it have been consumed, so it orders nothing else and does not
// wait for this thread's outstanding global stores.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t remote_bar) {
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote_bar) : "memory");
}

// Arm a local mbarrier for `bytes` of incoming asynchronous stores (one arrival, relaxed).
__device__ __forceinline__ void mbar_arm_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Cluster-wide barrier of all non-exited threads (release / acquire).  Used once after the
// mbarrier initialisation (no remote arrival may precede it) and once before exit (no CTA may
// leave while another can still touch its shared memory).
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Rounding-explicit pieces of the explicit time update u^{n+1} = G (2 u^n - a- u^{n-1} + rhs)
// (Sec. 2 scheme with the sponge).  Every product and sum is one IEEE operation written
// out, so the compiler cannot fuse them differently in different kernel instantiations:
// all 2D variants (one tile per CTA, pipelined, single- or multi-model) give the same bits.
__device__ __forceinline__ float leapfrog(float G, float c, float am, float prev, float rhs) {
    return __fmul_rn(G, __fadd_rn(__fmaf_rn(-am, prev, __fadd_rn(c, c)), rhs));
}

// G = 1 / (1 + e) and a- = 1 - e of a sponge cell; left at 1 where e = 0.
__device__ __forceinline__ void sponge_pair(float e, float& G, float& am) {
    if (e != 0.f) {
        G = __frcp_rn(__fadd_rn(1.f, e));
        am = __fsub_rn(1.f, e);
    }
}

// 3D tiled TMA load of one box into shared memory, completing on `bar`.
// The innermost coordinate x must be a multiple of 4 (16 bytes of FP32).
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* map, int x, int y,
                                            int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// 4D tiled TMA load (x, y, z, volume); same alignment rule on x.
__device__ __forceinline__ void tma_load_4d(void* smem_dst, const CUtensorMap* map, int x, int y, int z,
                                            int v, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(v), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void set_dev_error(int* err, int bit) {
    if (err) atomicOr(err, bit);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 ld4_stream(const float* p) {
    return __ldcs(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ float get(const float4& v, int j) {
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// Packed FP32x2 arithmetic on the lane pairs (0,1), (2,3) of a float4: each lane is rounded
// exactly as the scalar operation of the same name, so packed and scalar paths agree bit for bit.
struct P4 {
    float2 a, b;
};
__device__ __forceinline__ P4 p4(const float4& v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ P4 p4(float v0, float v1, float v2, float v3) {
    return {make_float2(v0, v1), make_float2(v2, v3)};
}
__device__ __forceinline__ float4 f4(const P4& p) { return make_float4(p.a.x, p.a.y, p.b.x, p.b.y); }
__device__ __forceinline__ float2 sub2(float2 x, float2 y) {  // x - y, one rounding
    return __ffma2_rn(y, make_float2(-1.f, -1.f), x);
}
__device__ __forceinline__ P4 p4add(const P4& x, const P4& y) { return {__fadd2_rn(x.a, y.a), __fadd2_rn(x.b, y.b)}; }
__device__ __forceinline__ P4 p4sub(const P4& x, const P4& y) { return {sub2(x.a, y.a), sub2(x.b, y.b)}; }
__device__ __forceinline__ P4 p4mul(const P4& x, const P4& y) { return {__fmul2_rn(x.a, y.a), __fmul2_rn(x.b, y.b)}; }
__device__ __forceinline__ P4 p4fma(const P4& x, const P4& y, const P4& z) {
    return {__ffma2_rn(x.a, y.a, z.a), __ffma2_rn(x.b, y.b, z.b)};
}
__device__ __forceinline__ P4 p4neg(const P4& x) {
    return {make_float2(-x.a.x, -x.a.y), make_float2(-x.b.x, -x.b.y)};
}
// leapfrog() of an interior cell (G = a- = 1): (2c - prev) + rhs; the factor G = 1 is exact.
__device__ __forceinline__ P4 p4leap1(const P4& c, const P4& prev, const P4& rhs) {
    return p4add(p4sub(p4add(c, c), prev), rhs);
}

// Bring the line holding p into L2 (a hint: no registers held, nothing returned).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Kahan-compensated s += v with running compensation c (explicit roundings).
__device__ __forceinline__ void kahan1(float& s, float& c, float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

__device__ __forceinline__ void kahan4(float4& s, float4& c, float v0, float v1, float v2, float v3) {
    kahan1(s.x, c.x, v0);
    kahan1(s.y, c.y, v1);
    kahan1(s.z, c.z, v2);
    kahan1(s.w, c.w, v3);
}

// a[j] += v for a runtime lane j of a 4-element register array (j outside 0..3: no-op).
// Written as an unrolled select so that the array stays in registers.
__device__ __forceinline__ void add_lane(float a[4], int j, float v) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k == j) a[k] += v;
}

// 8th-order central second-derivative weights w0..w4 (standard Taylor-series coefficients).
#define PROBE_W0 (-205.0 / 72.0)
#define PROBE_W1 (8.0 / 5.0)
#define PROBE_W2 (-1.0 / 5.0)
#define PROBE_W3 (8.0 / 315.0)
#define PROBE_W4 (-1.0 / 560.0)

}  // namespace probe
