// meta_persist.cu -- many registration problems of any shapes, 2-D and 3-D,
// T and sigma in ONE persistent kernel launch (arXiv:2106.08817: each problem
// is one cost_and_grad, Eq. 3 shooting in the semi-Lagrangian form of
// Sec. 2.3, the Eq. 4 cost and its adjoint), sm_103a.
//
// The launch sequence of each problem's call is recorded on the host (the
// launchers append a record instead of launching, meta_kernels.h) and becomes
// a list of phases, one per recorded launch, each with the tiles (CTAs) of
// that launch.  The phases of all problems are interleaved into one global
// order by each problem's progress (the fraction of its tiles done at the
// phase's midpoint), so the problems advance together and their phases fill
// the GPU side by side.  The kernel's CTAs take tiles from one atomic counter
// in that order; a tile first waits, with a bounded spin, until every tile of
// its problem's earlier phases has finished (a completion counter per
// problem), then runs the very body of the recorded kernel on a virtual block
// (VBlk), so every output is computed by the same code in the same order as
// by the ordinary launches: the results are bit for bit those of the separate
// calls.
//
// Progress without co-residency: tiles are taken in increasing order, and a
// tile only waits for tiles of earlier phases of its problem, whose indices
// are smaller.  The smallest unfinished tile therefore never waits, and its
// CTA is running; no assumption on how many CTAs are resident is needed.
//
// Memory ordering: a finished item is published after a block barrier by a
// gpu-scope release reduction on its problem's counter; a waiting item's
// thread 0 reads the counter with gpu-scope acquire loads (which also drop
// the SM's L1 lines, so later plain loads of the CTA see other CTAs' writes)
// before its CTA passes the block barrier.  Bodies read
// read-only data with plain loads here (ld_ro), tensor maps from the plan's
// table after a tensormap acquire fence, and order their TMA reads after the
// acquire with a proxy fence.
//
// Failure detection: a dependency wait that runs past its limit (5 s by
// default, or a test's shorter one) latches the timeout bit in the waiting
// problem's workspace status word and in the plan's status word, and raises
// an abort flag that every CTA checks before it takes another tile; nothing
// traps.  A body whose TMA wait ran out (its own bounded wait) latches its
// workspace's bit, as in an ordinary launch, and its tile still counts as
// done, so no other tile waits on it for ever.
#define META_BODIES_ONLY
#include "meta_blur.cu"
#include "meta_step.cu"
#include "meta_adjoint.cu"
#undef META_BODIES_ONLY

#include <algorithm>
#include <cstring>
#include <vector>

namespace meta {
namespace {

constexpr unsigned kPersistTimeout = 1u;  // a dependency wait ran out (results invalid)
constexpr int kPersistThreads = 256;

// One recorded launch of one problem, as the device reads it.
struct alignas(16) DPhase {
    int kind, ndim, sub, kc;
    int gx, gy, gz, bx, by;  // grid and block of the recorded launch
    int inst;                // problem index
    unsigned need;           // tiles of the problem's earlier phases
    int tm, taps;            // first tensor map, taps (indices into the tables; -1: none)
    int ntiles;              // tiles (CTAs) of the recorded launch
    int per;                 // tiles per work item (small tiles run in groups)
    long long first;         // global index of the phase's first work item
    PArgs a;
};

// Tiles per work item: the pointwise and 2-D tile kinds do little work per
// tile (32 x 8 or 32 x 16 voxels), so a work item runs several in a row.
int tiles_per_item(int kind, int ndim) {
    switch (kind) {
        case PK_PACK:
        case PK_ADJINIT:
        case PK_ADJREC:
            return 16;
        case PK_GRADP:
            return ndim == 3 ? 16 : 8;
        case PK_ADVECT:
        case PK_TRANS:
            return ndim == 3 ? 1 : 8;
        case PK_XPASS:
        case PK_STRIDED:
            return 4;
        default:
            return 1;
    }
}

// Control block of one plan: the work counter, per-launch abort flag, sticky
// status, and the completion counter of every problem.
struct Ctl {
    unsigned long long next;
    unsigned int abort;
    unsigned int status;
    unsigned int done[1];  // [n]
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// done += n with release semantics at gpu scope: the CTA's writes before the
// block barrier that precedes it are visible to whoever acquires the counter.
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned n) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(n) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
    return *reinterpret_cast<const volatile unsigned*>(p);
}

// Waits (bounded) until *cnt >= need; false if it ran out or the launch was
// abandoned meanwhile.
__device__ bool wait_done(const unsigned* cnt, unsigned need, Ctl* ctl,
                          unsigned long long limit_ns, unsigned* fault) {
    if (ld_acquire(cnt) >= need) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 0; it < (1u << 26); ++it) {
        __nanosleep(256);
        if (ld_acquire(cnt) >= need) return true;
        if ((it & 31u) == 31u) {
            if (ld_volatile(&ctl->abort)) return false;
            if (globaltimer_ns() - t0 > limit_ns) break;
        }
    }
    atomicOr(&ctl->status, kPersistTimeout);
    atomicExch(&ctl->abort, 1u);
    if (fault) atomicOr(fault, kFaultTmaTimeout);
    return false;
}

__device__ __forceinline__ void body_zero(const VBlk& kb, unsigned int* p, int n) {
    const int base = kb.bx() * 1024;
    for (int i = kb.tx(); i < 1024; i += kb.ndx())
        if (base + i < n) p[base + i] = 0u;
}

// The tap loops compiled into the persistent kernel: 2 to 5 chunks of 8 (sigma
// up to 6); other widths run the runtime loop, which sums the same products in
// the same order.
#define META_KC_CASES(F) \
    case 2: F(2); break; \
    case 3: F(3); break; \
    case 4: F(4); break; \
    case 5: F(5); break; \
    default: F(0); break;

template <int NDIM, bool GRADP>
__device__ __forceinline__ void run_xpass(const VBlk& kb, const DPhase& ph,
                                          const CUtensorMap* tms, const Taps* taps) {
    const PArgs& a = ph.a;
#define META_X(KC)                                                                            \
    body_xpass<VBlk, NDIM, GRADP, KC>(kb, tms[ph.tm], tms[ph.tm + 1], taps[ph.taps], a.g,    \
                                      a.i0, a.i1, a.c[0], a.i2, a.w[0], a.fault)
    switch (ph.kc) { META_KC_CASES(META_X) }
#undef META_X
}

template <int NDIM, int AXIS>
__device__ __forceinline__ void run_strided(const VBlk& kb, const DPhase& ph,
                                            const CUtensorMap* tms, const Taps* taps) {
    const PArgs& a = ph.a;
#define META_S(KC)                                                                            \
    body_strided<VBlk, NDIM, AXIS, KC>(kb, tms[ph.tm], taps[ph.taps], a.g, a.i0, a.i1,       \
                                       a.c[0], a.f0, a.w[0], a.fault)
    switch (ph.kc) { META_KC_CASES(META_S) }
#undef META_S
}

// Runs one tile of phase ph (in shared memory) on the virtual block kb.
__device__ void run_tile(const VBlk& kb, const DPhase& ph, const CUtensorMap* tms,
                         const Taps* taps) {
    const PArgs& a = ph.a;
    const bool d3 = ph.ndim == 3;
    switch (ph.kind) {
        case PK_ZERO:
            body_zero(kb, a.md, a.n);
            break;
        case PK_PACK:
            if (d3) body_pack<VBlk, 3>(kb, a.g, a.c[0], a.c[1], a.w[0], a.w[1]);
            else body_pack<VBlk, 2>(kb, a.g, a.c[0], a.c[1], a.w[0], a.w[1]);
            break;
        case PK_XPASS:
            if (d3) {
                if (ph.sub) run_xpass<3, true>(kb, ph, tms, taps);
                else run_xpass<3, false>(kb, ph, tms, taps);
            } else {
                if (ph.sub) run_xpass<2, true>(kb, ph, tms, taps);
                else run_xpass<2, false>(kb, ph, tms, taps);
            }
            break;
        case PK_STRIDED:
            if (!d3) run_strided<2, 0>(kb, ph, tms, taps);
            else if (ph.sub == 1) run_strided<3, 1>(kb, ph, tms, taps);
            else run_strided<3, 0>(kb, ph, tms, taps);
            break;
        case PK_ADVECT:
            if (d3)
                body_advect3d<VBlk, false>(kb, tms[ph.tm], tms[ph.tm + 1], a.g, a.cf, a.t, a.sl,
                                           a.zc, a.w[0], a.md, a.fault);
            else body_advect2d<VBlk, false>(kb, a.g, a.cf, a.t, a.sl, a.w[0], a.c[0], a.md);
            break;
        case PK_COSTP:
            if (d3) body_cost_partials<VBlk, 3>(kb, a.g, a.sl, a.c[0], a.c[1], a.c[2], a.d[0]);
            else body_cost_partials<VBlk, 2>(kb, a.g, a.sl, a.c[0], a.c[1], a.c[2], a.d[0]);
            break;
        case PK_ADJINIT:
            if (d3)
                body_adj_init<VBlk, 3, true>(kb, a.g, a.cf, a.sl, a.c[0], a.c[1], a.c[2], a.c[3],
                                             a.cmd, a.w[0], a.w[1], a.w[2], a.w[3], a.w[4]);
            else
                body_adj_init<VBlk, 2, true>(kb, a.g, a.cf, a.sl, a.c[0], a.c[1], a.c[2], a.c[3],
                                             a.cmd, a.w[0], a.w[1], a.w[2], a.w[3], a.w[4]);
            break;
        case PK_COSTF:
            body_cost_final<VBlk>(kb, a.n, a.cf, a.d[0], a.d[1]);
            break;
        case PK_ADJREC:
            if (d3)
                body_adj_records<VBlk, 3>(kb, a.g, a.cf, a.sl, a.c[0], a.c[1], a.c[2], a.c[3],
                                          a.w[0]);
            else
                body_adj_records<VBlk, 2>(kb, a.g, a.cf, a.sl, a.c[0], a.c[1], a.c[2], a.c[3],
                                          a.w[0]);
            break;
        case PK_TRANS:
            if (d3)
                body_adj_transport3d<VBlk>(kb, tms[ph.tm], tms[ph.tm + 1], tms[ph.tm + 2], a.g,
                                           a.cf, a.t, a.sl, a.zc, a.c[0], a.cmd, a.c[1], a.w[0],
                                           a.w[1], a.w[2], a.fault);
            else
                body_adj_transport2d<VBlk>(kb, a.g, a.cf, a.t, a.sl, a.c[0], a.cmd, a.c[1],
                                           a.w[0], a.w[1], a.w[2], a.fault);
            break;
        case PK_GRADP:
            if (d3)
                body_adj_gradp3_pair<VBlk>(kb, a.g, a.cf, a.t, a.mode, a.sl, a.c[0], a.c[1],
                                           a.cmd, a.c[2], a.w[0], a.w[1], a.w[2], a.w[3],
                                           a.w[4], a.w[5], a.w[6]);
            else
                body_adj_gradp2d<VBlk, false>(kb, a.g, a.cf, a.t, a.mode, a.sl, a.c[0], a.c[1],
                                              a.cmd, a.c[2], a.w[0], a.w[1], a.w[2], a.w[3],
                                              a.w[4], a.w[5], a.w[6]);
            break;
        default:
            break;
    }
}

// Copies the descriptor of phase ph into shared memory with asynchronous
// 16-byte copies (thread 0; waited for by cp.async.wait_all).
__device__ __forceinline__ void fetch_phase(DPhase* dst, const DPhase* src) {
    for (int i = 0; i < (int)(sizeof(DPhase) / 16); ++i)
        cp_async16(reinterpret_cast<char*>(dst) + 16 * i,
                   reinterpret_cast<const char*>(src) + 16 * i, true);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// hold >= 0 (self-test only): the first phase of problem `hold` never reports
// its tiles, so the problem's second phase waits until its limit runs out.
//
// Thread 0 keeps two items ahead of the tiles: while the CTA runs item k it
// has the index of item k+2 in flight, the descriptor of item k+1 landing in
// the other shared slot, and a first read of item k+1's dependency counter.
// A fetched item only starts after the CTA's current one has finished, so the
// progress argument above still holds (the CTA holding the smallest unfinished
// item has finished everything before it and runs it next).
__global__ void __launch_bounds__(kPersistThreads, 2)
k_persist(const DPhase* __restrict__ phases, const long long* __restrict__ firsts, int nph,
          long long total, const CUtensorMap* tms, const Taps* taps, Ctl* ctl,
          unsigned long long limit_ns, int hold) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ DPhase sph[2];
    __shared__ long long s_item[2];
    __shared__ int s_go;
    const int tid = threadIdx.x;
    // thread 0's pipeline: items cur (running), nx (next), nx2 (after next)
    int ph = 0;  // phase of the latest item scanned (items come in increasing order)
    long long nx = 0;
    unsigned long long nx2 = 0;
    unsigned early = 0;  // first read of the next item's dependency counter
    auto scan = [&](long long it) {
        while (ph + 1 < nph && firsts[ph + 1] <= it) ++ph;
        return ph;
    };
    if (tid == 0) {
        const long long it = (long long)atomicAdd(&ctl->next, 1ull);
        int go = it < total;
        if (go) {
            const int p0 = scan(it);
            fetch_phase(&sph[0], phases + p0);
            go = wait_done(&ctl->done[phases[p0].inst], phases[p0].need, ctl, limit_ns,
                           phases[p0].a.fault);
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        s_item[0] = it;
        s_go = go;
        nx = (long long)atomicAdd(&ctl->next, 1ull);
        nx2 = atomicAdd(&ctl->next, 1ull);
    }
    __syncthreads();
    for (int k = 0; s_go; ++k) {
        const int slot = k & 1;
        const DPhase& P = sph[slot];
        if (tid == 0 && nx < total) {  // the next item: descriptor and a first dependency read
            const int pn = scan(nx);
            fetch_phase(&sph[slot ^ 1], phases + pn);
            early = ld_relaxed(&ctl->done[phases[pn].inst]);  // no ordering: the tiles go on
        }
        const int t0 = (int)(s_item[slot] - P.first) * P.per;
        const int t1 = min(t0 + P.per, P.ntiles);
        VBlk kb;
        kb.nthr = P.bx * P.by;
        // the 3-D gradp tiles (128 threads, no barrier, no shared memory) run two
        // at a time, one per half of the CTA
        const int lanes = (P.kind == PK_GRADP && P.ndim == 3 && 2 * kb.nthr <= kPersistThreads)
                              ? 2 : 1;
        const int sub = tid / kb.nthr, ltid = tid - sub * kb.nthr;
        kb.tx_ = ltid % P.bx;
        kb.ty_ = ltid / P.bx;
        kb.ndx_ = P.bx;
        kb.gx_ = P.gx;
        const int gxy = P.gx * P.gy;
        for (int t = t0; t < t1; t += lanes) {
            const int tt = t + sub;
            kb.bz_ = tt / gxy;
            const int r = tt - kb.bz_ * gxy;
            kb.by_ = r / P.gx;
            kb.bx_ = r - kb.by_ * P.gx;
            if (sub < lanes && tt < t1) run_tile(kb, P, tms, taps);
            if (t + lanes < t1) __syncthreads();  // the next tile reuses the shared memory
        }
        __syncthreads();
        if (tid == 0) {
            // publish this item's tiles (release at gpu scope, after the barrier)
            if (!(P.inst == hold && P.need == 0u))
                red_release_add(&ctl->done[P.inst], (unsigned)(t1 - t0));
            int go = nx < total;
            if (go) {
                // the next item's phase (scanned above): its dependencies were read before
                // this item's tiles; if they were met, a fence makes that read an acquire
                // (it also drops the SM's L1 lines), else wait with acquire loads
                const DPhase& N = phases[ph];
                if (early < N.need)
                    go = wait_done(&ctl->done[N.inst], N.need, ctl, limit_ns, N.a.fault);
                else
                    asm volatile("fence.acq_rel.gpu;" ::: "memory");
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            s_item[slot ^ 1] = nx;
            s_go = go;
            nx = (long long)nx2;
            nx2 = atomicAdd(&ctl->next, 1ull);  // in flight during the next item
        }
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------- host side

struct PersistPlan {
    DPhase* phases = nullptr;
    long long* firsts = nullptr;
    CUtensorMap* tms = nullptr;
    Taps* taps = nullptr;
    Ctl* ctl = nullptr;
    size_t ctl_bytes = 0;
    int nph = 0, ninst = 0, grid = 0;
    long long total = 0;
    size_t smem = 0;
};

void persist_free(PersistPlan* p) {
    if (!p) return;
    cudaFree(p->phases);
    cudaFree(p->firsts);
    cudaFree(p->tms);
    cudaFree(p->taps);
    cudaFree(p->ctl);
    delete p;
}

cudaError_t persist_build(const std::vector<std::vector<PRec>>& recs, PersistPlan** out) {
    *out = nullptr;
    const int n = (int)recs.size();
    std::vector<DPhase> all;
    std::vector<CUtensorMap> tms;
    std::vector<Taps> taps;
    struct Key {
        double key;
        int inst, k;
    };
    std::vector<Key> order;
    std::vector<std::vector<DPhase>> per(n);
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        // this problem's tensor maps and taps, each stored once
        std::vector<int> tm_idx, tap_idx;
        long long tiles_i = 0;
        for (const PRec& e : recs[i]) {
            if (e.bx * e.by > kPersistThreads || e.bx * e.by <= 0 || (e.bx * e.by) % 32 != 0)
                return cudaErrorNotSupported;
            DPhase d;
            std::memset(&d, 0, sizeof(d));
            d.kind = e.kind;
            d.ndim = e.ndim;
            d.sub = e.sub;
            d.kc = e.kc;
            d.gx = (int)e.grid.x;
            d.gy = (int)e.grid.y;
            d.gz = (int)e.grid.z;
            d.bx = e.bx;
            d.by = e.by;
            d.inst = i;
            d.ntiles = d.gx * d.gy * d.gz;
            d.per = tiles_per_item(e.kind, e.ndim);
            d.a = e.a;
            d.tm = -1;
            d.taps = -1;
            if (e.ntm > 0) {
                d.tm = (int)tms.size();
                for (int k = 0; k < e.ntm; ++k) tms.push_back(e.tm[k]);
            }
            if (e.has_taps) {
                int found = -1;
                for (int k : tap_idx)
                    if (std::memcmp(&taps[k], &e.taps, sizeof(Taps)) == 0) found = k;
                if (found < 0) {
                    found = (int)taps.size();
                    taps.push_back(e.taps);
                    tap_idx.push_back(found);
                }
                d.taps = found;
            }
            smem = std::max(smem, e.smem);
            per[i].push_back(d);
            tiles_i += d.ntiles;
        }
        long long acc = 0;
        for (int k = 0; k < (int)per[i].size(); ++k) {
            per[i][k].need = (unsigned)acc;
            const double mid = (double)acc + 0.5 * per[i][k].ntiles;
            order.push_back({mid / (double)std::max(1LL, tiles_i), i, k});
            acc += per[i][k].ntiles;
        }
        if (acc >= (1LL << 31)) return cudaErrorNotSupported;
    }
    std::sort(order.begin(), order.end(), [](const Key& a, const Key& b) {
        if (a.key != b.key) return a.key < b.key;
        if (a.inst != b.inst) return a.inst < b.inst;
        return a.k < b.k;
    });
    long long first = 0;
    std::vector<long long> firsts;
    for (const Key& o : order) {
        DPhase d = per[o.inst][o.k];
        d.first = first;
        firsts.push_back(first);
        first += (d.ntiles + d.per - 1) / d.per;  // work items of the phase
        all.push_back(d);
    }
    PersistPlan* p = new PersistPlan();
    p->nph = (int)all.size();
    p->ninst = n;
    p->total = first;
    p->smem = std::max(smem, (size_t)256);
    cudaError_t e = cudaMalloc(&p->phases, sizeof(DPhase) * std::max<size_t>(1, all.size()));
    if (e == cudaSuccess)
        e = cudaMalloc(&p->firsts, sizeof(long long) * std::max<size_t>(1, firsts.size()));
    if (e == cudaSuccess)
        e = cudaMalloc(&p->tms, sizeof(CUtensorMap) * std::max<size_t>(1, tms.size()));
    if (e == cudaSuccess) e = cudaMalloc(&p->taps, sizeof(Taps) * std::max<size_t>(1, taps.size()));
    p->ctl_bytes = sizeof(Ctl) + sizeof(unsigned) * (size_t)n;
    if (e == cudaSuccess) e = cudaMalloc(&p->ctl, p->ctl_bytes);
    if (e == cudaSuccess && !all.empty())
        e = cudaMemcpy(p->phases, all.data(), sizeof(DPhase) * all.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !firsts.empty())
        e = cudaMemcpy(p->firsts, firsts.data(), sizeof(long long) * firsts.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tms.empty())
        e = cudaMemcpy(p->tms, tms.data(), sizeof(CUtensorMap) * tms.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !taps.empty())
        e = cudaMemcpy(p->taps, taps.data(), sizeof(Taps) * taps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->ctl, 0, p->ctl_bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p->smem);
    int per_sm = 0, dev = 0, nsm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, kPersistThreads,
                                                          p->smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e != cudaSuccess) {
        persist_free(p);
        return e;
    }
    p->grid = (int)std::min<long long>((long long)per_sm * nsm, std::max(1LL, p->total));
    *out = p;
    return cudaSuccess;
}

// One launch: clear the counters (not the sticky status), then the kernel.
cudaError_t persist_launch(PersistPlan* p, cudaStream_t st, unsigned long long limit_ns,
                           int hold) {
    cudaError_t e = cudaMemsetAsync(p->ctl, 0, offsetof(Ctl, status), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(reinterpret_cast<char*>(p->ctl) + offsetof(Ctl, done), 0,
                        sizeof(unsigned) * (size_t)p->ninst, st);
    if (e != cudaSuccess) return e;
    k_persist<<<p->grid, kPersistThreads, p->smem, st>>>(p->phases, p->firsts, p->nph, p->total,
                                                          p->tms, p->taps, p->ctl, limit_ns, hold);
    return cudaGetLastError();
}

// The plan's sticky status word (bit 0: a dependency wait ran out).
cudaError_t persist_status(PersistPlan* p, int clear, cudaStream_t st, unsigned* bits) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(bits, &p->ctl->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    *bits &= kPersistTimeout;
    if (clear) {
        e = cudaMemsetAsync(&p->ctl->status, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e;
}

int persist_problems(const PersistPlan* p) { return p->ninst; }
long long persist_tiles(const PersistPlan* p) { return p->total; }
int persist_grid(const PersistPlan* p) { return p->grid; }

}  // namespace meta
