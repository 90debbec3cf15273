// meta_common.cuh -- shared definitions of the sm_103a semi-Lagrangian
// Metamorphosis kernels: geometry, tap tables, TMA / mbarrier helpers in
// inline PTX, the relative-coordinate foot computation and the workspace map.
#pragma once

#include <cmath>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

namespace meta {

// ---------------------------------------------------------------- limits
constexpr int kMaxTaps = 128;  // padded tap table length (r <= 54)
constexpr int kMaxR = 54;      // sigma <= 18
constexpr int kBX = 8;         // x-pass: outputs per thread along x
constexpr int kTX = 128;       // x-pass: largest tile width along x
constexpr int kRows = 16;      // x-pass: rows per CTA (2-D: 16 y; 3-D: 4 z x 4 y)
constexpr int kBA = 16;        // strided pass: outputs per thread along the axis
constexpr int kTA = 128;       // strided pass: largest built-in tile length along the axis
constexpr int kTAMax = 192;    // strided pass: largest tuned tile length (L + taps <= 256, one TMA box)
constexpr int kTXS = 32;       // strided pass: columns per CTA
// strided pass: one thread per column pair and group of kBA outputs along the
// axis (L / kBA groups of 16 threads), rounded up to whole warps
inline int strided_threads(int L) { return (L / kBA * (kTXS / 2) + 31) / 32 * 32; }

// Tiles of a blur pass split an extent n into ceil(n / maxlen) equal tiles,
// each rounded up to a multiple of q, so that no CTA carries a mostly empty
// tail tile (160 = 2 x 80 rather than 128 + 32).
inline int even_tile(int n, int maxlen, int q) {
    const int nt = (n + maxlen - 1) / maxlen;
    const int l = (n + nt - 1) / nt;
    return (l + q - 1) / q * q;
}

// x halo of the x pass for kernel radius r (r4 = r rounded up to 4): the
// smallest multiple of 4 that (a) keeps every column a nonzero tap reaches at
// least one column inside the staged row (its x neighbours are staged for the
// gradient of m), (b) starts each output's tap window inside the row (>= r4) and
// (c) ends the last thread's window of kp = roundup(r4 + r + 1, 8) taps inside
// it.
__host__ __device__ constexpr int xpass_hx(int r, int r4) {
    const int kp = (r4 + r + 1 + 7) / 8 * 8;
    const int a = r + 1, c = kp - r4;
    const int m = a > r4 ? (a > c ? a : c) : (r4 > c ? r4 : c);
    return (m + 3) / 4 * 4;
}

// Staged row length of the x pass for tile width txw: txw + 2 hx, plus 4 pad
// columns where the TMA box allows, so that the row stride in 16-byte units is
// odd and two rows read by one quarter-warp hit all eight 16-byte bank groups.
__host__ __device__ constexpr int xpass_lw(int txw, int r, int r4) {
    return txw + 2 * xpass_hx(r, r4) + ((txw + 2 * xpass_hx(r, r4) + 4 <= 256) ? 4 : 0);
}

// Threads of an x-pass CTA: kRows rows of txw / 8 threads, padded to a
// multiple of 4 per row (conflict-free 16-byte loads in the blur phase).
__host__ __device__ constexpr int xpass_threads(int txw) {
    return ((txw / kBX + 3) & ~3) * kRows;
}

// Largest staged row of the x pass: the TMA box limit of 256 elements.
constexpr int kMaxLW = 256;

// The max displacement of step t, instance b lives at maxdisp[kMaxdispStride *
// (t * B + b)]: one 128-byte line per slot, so that the per-CTA atomics of
// different instances do not queue on one L2 line.
constexpr int kMaxdispStride = 32;

// Rows of a 3-D advect CTA's column (two per thread); its staged window has a
// one-row halo on each side.
constexpr int kAdvRows = 12;
// Rows of a 3-D transport CTA's column (two nodes per thread, so 32 x kTransRows / 2
// threads); its staged windows have a one-row halo on each side.
constexpr int kTransRows = 8;

// Fault / information bits latched in the workspace header.
constexpr unsigned kFaultTmaTimeout = 1u;  // a bounded TMA wait ran out (fault)
constexpr unsigned kInfoScatter = 2u;      // adjoint used the atomic scatter (large steps)
constexpr unsigned kFaultBounds = 4u;      // bounds-checked build: an index left its range

// ---------------------------------------------------------------- geometry
// An instance is an (nz,) ny x nx grid stored with row pitch P floats
// (P = nx rounded up to a multiple of 4, so that every row starts on a 16-byte
// boundary as TMA requires).  For 2-D problems nz = 1.
struct Geom {
    int nz, ny, nx;   // extents (nz = 1 in 2-D)
    int P;            // row pitch in floats
    long long slab;   // ny * P
    long long inst;   // nz * ny * P  (floats per instance slice)
    int B;            // batch
    int nT;           // time steps T
    int txw;          // x-pass tile width (multiple of kBX, <= kTX)
    int ly, lz;       // strided-pass tile lengths along y and z (multiples of kBA, <= kTAMax)
    int zct, zca;     // planes per CTA of the 3-D transport / advect (0: heuristic)
    unsigned nyt_mul; // ceil(2^32 / nyt), nyt = ceil(ny / 8): q = umulhi(n, nyt_mul) = n / nyt
                      // exactly for n * nyt < 2^32 (n < 65536, nyt <= 8192); 0 when nyt = 1
    unsigned int* chk;  // the workspace status word (bounds-checked build: kFaultBounds)
};

// Bounds-checked build (META_CHECK_BOUNDS): v must lie in [lo, hi]; otherwise the
// bounds bit is latched in the workspace status word and v is clamped into the
// range, so that the access it indexes stays inside its buffer.  In the ordinary
// build it returns v and costs nothing.
__device__ __forceinline__ int chk_range(const Geom& g, int v, int lo, int hi) {
#ifdef META_CHECK_BOUNDS
    if (v < lo || v > hi) {
        if (g.chk) atomicOr(g.chk, kFaultBounds);
        v = v < lo ? lo : hi;
    }
#else
    (void)g;
    (void)lo;
    (void)hi;
#endif
    return v;
}

// n / nyt for a grid index n of the pointwise kernels (see Geom::nyt_mul).
__device__ __forceinline__ int div_nyt(const Geom& g, int n) {
    return g.nyt_mul ? (int)__umulhi((unsigned)n, g.nyt_mul) : n;
}

// Planes per CTA of a kernel that marches along z over 32 x 8 columns: the
// chunk that best trades the `halo` extra planes each chunk stages against
// the fill of the last wave (ctas_per_sm resident CTAs per SM).
inline int march_chunk(const Geom& g, int ctas_per_sm, int halo, int rows = 8) {
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            nsm <= 0)
            nsm = 152;
    }
    const long long cols = (long long)((g.nx + 31) / 32) * ((g.ny + rows - 1) / rows) * g.B;
    const int cand[] = {4, 6, 8, 12, 16, 24, 32};
    int best = 8;
    double best_s = -1.0;
    for (int zc : cand) {
        const int nch = (g.nz + zc - 1) / zc;
        const double waves = (double)(cols * nch) / ((double)ctas_per_sm * nsm);
        const double fill = waves / std::ceil(waves);
        const double zr = (double)g.nz / nch;  // planes per chunk
        const double s = fill * zr / (zr + halo);
        if (s > best_s + 1e-9) {
            best_s = s;
            best = zc;
        }
    }
    return best;
}

__host__ __device__ inline long long gidx(const Geom& g, int z, int y, int x) {
    return (long long)z * g.slab + (long long)y * g.P + x;
}

// Gaussian taps passed by value (constant bank, uniform reads).
struct Taps {
    int r;       // radius ceil(3 sigma)
    int kp;      // taps in the loop, multiple of 8 (zero padded)
    int r4;      // x-pass: radius rounded up to a multiple of 4
    float w[kMaxTaps];
};

// Slot indices of the times a launch touches.  A state slot holds one (I, p)
// pair of the trajectory buffer (slices (2 slot + f) B + b), a u slot one u_t
// (slices (slot d + a) B + b).  Keeping every state, slot = time; with step
// checkpointing the host maps times onto checkpoint and segment slots.
struct Slots {
    int st;   // state of time t (input)
    int st1;  // advect: state of t+1 (output); adjoint: state of the record's time
    int ut;   // u of step t
    int ut1;  // adjoint: u of the record's time
    int s0;   // state of time 0
    int u0;   // u of step 0
    int sT;   // state of time T
};

// Per-launch scalars of the scheme.
struct Coefs {
    const float* mu;      // [B]
    const float* rho;     // [B]
    const float* lambda;  // [B]
    float dt;             // 1/T
    int pdet;             // momentum update: 0 p~ (1 - dt div v), 1 p~ det(Id - dt Dv)
    int scheme;           // 0 semi-Lagrangian, 1 Eulerian, 2 hybrid
};

// ------------------------------------------------- relative-coordinate foot
// Foot of voxel c displaced by d (y = c + d), clamped to [0, n-1].  Computed
// from the displacement rather than from the absolute coordinate so that
// sub-ulp displacements keep their sign in FP32.  i0 = floor(y) lowered to
// n-2 at the far edge, f = y - i0 in [0, 1], inside = clamp inactive.
struct Foot1 {
    int i0;
    float f;
    bool inside;
};

__device__ __forceinline__ Foot1 foot1(int c, float d, int n) {
    Foot1 r;
    const float lo = -(float)c;           // y <= 0      <=> d <= -c
    const float hi = (float)(n - 1 - c);  // y >= n - 1  <=> d >= n-1-c
    if (d <= lo) {
        r.i0 = 0;
        r.f = 0.f;
        r.inside = false;
    } else if (d >= hi) {
        r.i0 = n - 2;
        r.f = 1.f;
        r.inside = false;
    } else {
        const float fl = floorf(d);
        r.i0 = c + (int)fl;
        r.f = d - fl;
        r.inside = true;
    }
    return r;
}

// foot1 with the lower corner checked (bounds-checked build) against [0, n - 2],
// the range every interpolation at a foot indexes.
__device__ __forceinline__ Foot1 foot1g(const Geom& g, int c, float d, int n) {
    Foot1 r = foot1(c, d, n);
    r.i0 = chk_range(g, r.i0, 0, n - 2);
    return r;
}

// ----------------------------------------------------------- PTX helpers
// Two independent FP32 fused multiply-adds in one instruction (fma.rn.f32x2,
// sm_100 and later): lane k of the result is fmaf(a.k, b.k, c.k), rounded
// exactly as the scalar fmaf.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)),
          "l"(*reinterpret_cast<unsigned long long*>(&b)),
          "l"(*reinterpret_cast<unsigned long long*>(&c)));
    return *reinterpret_cast<float2*>(&d);
}
// Two FP32 products in one instruction (mul.rn.f32x2), lane k = a.k * b.k.
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)),
          "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&d);
}
// Two FP32 sums / differences in one instruction (add.rn.f32x2, sub.rn.f32x2),
// each lane rounded as the scalar __fadd_rn / __fsub_rn.
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)),
          "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&d);
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)),
          "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return *reinterpret_cast<float2*>(&d);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One try_wait; the thread may be suspended for up to 100 us (suspend-time
// hint) while the phase is still pending, so waiting warps take few issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on phase `parity`: gives up after limit_ns (2 s by default; or
// 2^24 polls), latches kFaultTmaTimeout in *fault and returns false.  A TMA
// copy that completes normally takes microseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned int* fault,
                                                  uint64_t limit_ns = 2000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15u) == 15u && globaltimer_ns() - t0 > limit_ns) break;
    }
    atomicOr(fault, kFaultTmaTimeout);
    return false;
}

// Tiled TMA loads into shared memory, completion counted on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
        "r"(smem_u32(bar))
        : "memory");
}

// A tensor map that lives in global memory (the persistent kernel's table,
// written by the host before the launch) is made visible to the TMA unit by an
// acquire fence of the tensormap proxy, once per thread that issues copies
// with it.  Tensor maps passed as kernel parameters need none.
__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}
// Orders this thread's earlier generic-proxy accesses to global memory (and
// those it has acquired from other CTAs) before its later async-proxy (TMA)
// accesses.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Ends an mbarrier's life, so that its shared memory may be reused (the next
// tile of the persistent kernel may run a body that stores data there).
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Plain arrival (no transaction bytes): completes the phase of a barrier
// initialised with count 1 when no copy is issued for it.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Load a box whose innermost coordinate is x, at (x, y[, z], slice).
template <int NDIM>
__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* map, uint64_t* bar,
                                             int x, int y, int z, int slice) {
    if constexpr (NDIM == 2)
        tma_load_3d(dst, map, bar, x, y, slice);
    else
        tma_load_4d(dst, map, bar, x, y, z, slice);
}

// Programmatic dependent launch: a kernel launched with the
// programmatic-serialization attribute may start while its predecessor in the
// stream finishes.  pdl_wait() blocks until the predecessor has completed and
// its writes are visible, so every kernel calls it before reading anything the
// previous kernel wrote.  No kernel signals its dependents early
// (griddepcontrol.launch_dependents): each CTA counts as signalled when it exits,
// so the successor's CTAs take SM slots only while the predecessor's last CTAs
// finish.  Signalled at the start of every CTA, they were resident and waiting
// during the predecessor's later waves, whose CTAs then had fewer slots: a
// 160x192x160 call took 9.64 ms that way against 9.04 ms.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Block context of a kernel body.  The bodies of the kernels read their block
// and thread indices, block and grid shapes, barriers and dynamic shared memory
// through it, so that one body serves two launch forms:
//  * HwBlk: an ordinary launch, everything from the hardware built-ins (the
//    generated code is that of a plain kernel);
//  * VBlk: one tile of a launch replayed inside the persistent kernel
//    (meta_persist.cu), whose CTA runs the tiles of many launches one after
//    another: indices and shapes are the replayed launch's, and the barrier is
//    the named barrier 1 over the first nthr threads (the tile's threads; the
//    persistent CTA may have more).
struct HwBlk {
    static constexpr bool kPersistent = false;
    // the dynamic shared memory of the launch (by symbol: its address is a
    // constant of the kernel, which keeps shared addressing cheap)
    __device__ __forceinline__ unsigned char* smem() const {
        extern __shared__ __align__(128) unsigned char meta_dyn_smem[];
        return meta_dyn_smem;
    }
    // unsigned, as the built-ins: index arithmetic (a division by a runtime tile
    // count, say) stays unsigned and on the uniform datapath
    __device__ __forceinline__ unsigned bx() const { return blockIdx.x; }
    __device__ __forceinline__ unsigned by() const { return blockIdx.y; }
    __device__ __forceinline__ unsigned bz() const { return blockIdx.z; }
    __device__ __forceinline__ unsigned tx() const { return threadIdx.x; }
    __device__ __forceinline__ unsigned ty() const { return threadIdx.y; }
    __device__ __forceinline__ unsigned ndx() const { return blockDim.x; }
    __device__ __forceinline__ unsigned gx() const { return gridDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int sync_or(int p) const { return __syncthreads_or(p); }
};

struct VBlk {
    int bx_, by_, bz_, tx_, ty_, ndx_, gx_, nthr;
    static constexpr bool kPersistent = true;
    __device__ __forceinline__ unsigned char* smem() const {
        extern __shared__ __align__(128) unsigned char meta_dyn_smem[];
        return meta_dyn_smem;
    }
    __device__ __forceinline__ unsigned bx() const { return (unsigned)bx_; }
    __device__ __forceinline__ unsigned by() const { return (unsigned)by_; }
    __device__ __forceinline__ unsigned bz() const { return (unsigned)bz_; }
    __device__ __forceinline__ unsigned tx() const { return (unsigned)tx_; }
    __device__ __forceinline__ unsigned ty() const { return (unsigned)ty_; }
    __device__ __forceinline__ unsigned ndx() const { return (unsigned)ndx_; }
    __device__ __forceinline__ unsigned gx() const { return (unsigned)gx_; }
    __device__ __forceinline__ void sync() const {
        asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
    }
    __device__ __forceinline__ int sync_or(int p) const {
        int r;
        asm volatile(
            "{\n\t.reg .pred q, s;\n\t"
            "setp.ne.s32 q, %1, 0;\n\t"
            "bar.red.or.pred s, 1, %2, q;\n\t"
            "selp.s32 %0, 1, 0, s;\n\t}"
            : "=r"(r)
            : "r"(p), "r"(nthr)
            : "memory");
        return r;
    }
};

// Read-only global load: through the non-coherent cache in an ordinary launch;
// a plain load in the persistent kernel, whose buffers change between tiles
// (its gpu-scope acquire invalidates L1 before a tile reads another's output).
template <class K>
__device__ __forceinline__ float ld_ro(const float* p) {
    if constexpr (K::kPersistent) return *p;
    else return __ldg(p);
}

// 16-byte read-only load: through the non-coherent path in an ordinary launch,
// plain in the persistent kernel (its inputs may be written by other CTAs of
// the same launch).
template <class K>
__device__ __forceinline__ float4 ld4_ro(const float* p) {
    if constexpr (K::kPersistent) return *reinterpret_cast<const float4*>(p);
    else return __ldg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ float4 lds4(const float* p) {
    return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ float2 lds2(const float* p) {
    return *reinterpret_cast<const float2*>(p);
}

// PDL is on unless the environment sets META_NO_PDL=1 (read once).
inline bool pdl_enabled() {
    static const bool on = [] {
        const char* e = getenv("META_NO_PDL");
        return !(e && e[0] == '1');
    }();
    return on;
}

// Launches `kern` on `st` with the programmatic-serialization attribute.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

#define META_CHECK_LAUNCH(x)                    \
    do {                                        \
        const cudaError_t _e = (x);             \
        if (_e != cudaSuccess) return _e;       \
    } while (0)

}  // namespace meta
