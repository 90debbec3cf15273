// meta_blur.cu -- the Gaussian RKHS kernel K (Sec. 2.1 of arXiv:2106.08817)
// as separable 1-D passes, sm_103a.
//
//  * k_xpass<NDIM, GRADP>: pass along the contiguous axis x.  With GRADP it is
//    fused with the momentum field of Eq. 3: it stages I and p tiles (with a
//    one-voxel halo in y/z for the central differences) by TMA, forms
//    m_i = p * D_i I in shared memory, and blurs every component along x.
//    Without GRADP it blurs one component field.
//  * k_strided<NDIM, AXIS>: pass along a strided axis (y, or z in 3-D): a
//    column tile with an r-voxel halo is staged by one TMA load; the
//    out-of-bounds fill of TMA supplies the zero padding of K.
//
// Every thread produces consecutive outputs (8 along x, 16 along a strided
// axis) from a register window loaded once from shared memory, so each loaded
// value feeds up to that many FMAs.  With KC chunks of 8 taps known at compile
// time the outputs are computed in pairs by packed FP32 FMAs (fma.rn.f32x2,
// each lane the scalar fmaf in the same order).  Tiles split each extent into
// equal parts (Geom::txw, ly, lz).  No tensor cores: a banded Toeplitz product
// of 37 taps over 4-12 bytes per voxel is not a dense contraction.
#include "meta_kernels.h"

namespace meta {

// KC > 0: the tap loop has KC chunks of 8 at compile time (fully unrolled,
// taps read as immediate constant-bank operands); KC = 0: runtime taps.kp.
template <class K, int NDIM, bool GRADP, int KC>
__device__ __forceinline__ void body_xpass(const K& kb, const CUtensorMap& tmI, const CUtensorMap& tmP, const Taps& taps, Geom g, int sliceI, int sliceP, const float* pin, int out_slice0, float* __restrict__ out, unsigned int* fault) {
    unsigned char* smem_raw = kb.smem();
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float* base = reinterpret_cast<float*>(smem_raw + 128);

    const int HX = xpass_hx(taps.r, taps.r4);          // x halo (multiple of 4)
    const int LW = xpass_lw(g.txw, taps.r, taps.r4);   // staged row length
    const int rowsI = (NDIM == 2) ? (kRows + 2) : 36;
    const int tid = kb.tx();
    const int x0 = kb.bx() * g.txw;
    int y0, z0;
    if constexpr (NDIM == 2) {
        y0 = kb.by() * kRows;
        z0 = 0;
    } else {
        const int nty = (g.ny + 3) / 4;
        y0 = (kb.by() % nty) * 4;
        z0 = (kb.by() / nty) * 4;
    }
    // GRADP: one CTA per instance b = kb.bz().  Plain: one CTA per slice.
    const int b = GRADP ? (int)kb.bz() : (int)(kb.bz() % g.B);

    // sub-buffers start on 128-byte boundaries (TMA destinations)
    float* sI = base;
    float* sM = GRADP ? sI + ((rowsI * LW + 31) & ~31) : base;

    __shared__ int s_fail;  // ordinary launch: a wait for the tiles ran out
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        s_fail = 0;
    }
    kb.sync();
    if (tid == 0) {
        if constexpr (K::kPersistent) {
            tmap_acquire(&tmI);
            if (GRADP) tmap_acquire(&tmP);
            fence_proxy_async_global();
        }
        if constexpr (GRADP) {
            mbar_arrive_expect_tx(bar, (uint32_t)(rowsI * LW * 4));
            tma_load_box<NDIM>(sI, &tmI, bar, x0 - HX, y0 - 1, z0 - 1, sliceI + b);
        } else {
            mbar_arrive_expect_tx(bar, (uint32_t)(kRows * LW * 4));
            tma_load_box<NDIM>(sM, &tmI, bar, x0 - HX, y0, z0, sliceI + (int)kb.bz());
        }
    }
    // GRADP: items of four columns of one staged row (m is formed below).  Item idx
    // -> row and first column; idx < 2^12, so the rounded float quotient is the
    // exact integer one.
    const int LW4 = LW / 4;
    const int total = kRows * LW4;
    const float inv_lw4 = 1.f / (float)LW4;
    auto item_row = [&](int idx) { return (int)(((float)idx + 0.5f) * inv_lw4); };
    // p at an item's four columns, read from global memory (not staged: the shared
    // memory it would take keeps a third CTA off the SM); an item lies wholly inside
    // or wholly outside the pitched row
    auto load_p = [&](int idx) {
        float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const int row = item_row(idx);
        const int c = 4 * (idx - row * LW4);
        const int y = y0 + ((NDIM == 2) ? row : (row & 3));
        const int z = z0 + ((NDIM == 2) ? 0 : (row >> 2));
        const int xs = x0 - HX + c;
        if (idx < total && y < g.ny && z < g.nz && xs >= 0 && xs < g.P)
            p4 = ld4_ro<K>(pin + (long long)(sliceP + b) * g.inst + gidx(g, z, y, xs));
        return p4;
    };
    // the p of the thread's first kPre items is requested before the wait for the
    // I tile, so that the two latencies overlap
    constexpr int kPre = 3;
    float4 pre[kPre];
#pragma unroll
    for (int i = 0; i < kPre; ++i) pre[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (GRADP) {
#pragma unroll
        for (int i = 0; i < kPre; ++i) pre[i] = load_p(i * (int)kb.ndx() + tid);
    }

    // Ordinary launch: every warp waits (bounded) itself and goes on as soon as the
    // tiles have landed; a wait that runs out raises s_fail, which every thread reads
    // after the barrier that ends the gradient phase (the plain pass has no later
    // barrier, so its warps just leave).  Persistent kernel: warp 0 waits while the
    // others sleep in the barrier, and the barrier is retired before the next tile.
    if constexpr (K::kPersistent) {
        bool landed = true;
        if (tid < 32) landed = mbar_wait_bounded(bar, 0, fault);
        if (kb.sync_or(!landed)) return;
        if (tid == 0) mbar_inval(bar);  // every wait on it has returned
    } else {
        if (!mbar_wait_bounded(bar, 0, fault)) {
            if constexpr (!GRADP) return;
            s_fail = 1;  // still takes part in the gradient phase's shuffles (reads are
        }                // in bounds), then leaves with the others after its barrier
    }

    const int ncomp = GRADP ? NDIM : 1;
    if constexpr (GRADP) {
        // m_i = p * D_i I on the whole staged row range, four columns per
        // thread (finite everywhere; columns 0 and LW-1 only ever meet zero
        // taps, and there the missing neighbour is replaced by the column itself).
        const int lane = tid & 31;
        // the CTA has txw / 8 x 16 threads, so its last warp may hold 16 lanes
        const int wlast = min(31, (int)kb.ndx() - 1 - (tid & ~31));
        const unsigned wmask = wlast == 31 ? 0xffffffffu : ((2u << wlast) - 1u);
        auto form = [&](int base, const float4 p4) {
            const int idx = min(base + tid, total - 1);  // lanes past the end repeat the last
            const int row = item_row(idx);
            const int c = 4 * (idx - row * LW4);
            const int ty = (NDIM == 2) ? row : (row & 3);
            const int tz = (NDIM == 2) ? 0 : (row >> 2);
            const int y = y0 + ty, z = z0 + tz;
            const int rI = (NDIM == 2) ? (ty + 1) : ((tz + 1) * 6 + ty + 1);
            const float* Ir = sI + rI * LW;
            const float4 ic = lds4(Ir + c);
            // columns c - 1 and c + 4 from the neighbouring lanes (same row whenever
            // the column exists; the lanes at the warp's two ends read them), instead
            // of scalar loads at a 16-byte stride (four-way bank conflicts)
            float left = __shfl_up_sync(wmask, ic.w, 1);
            float right = __shfl_down_sync(wmask, ic.x, 1);
            if (lane == 0 && c > 0) left = Ir[c - 1];
            if (lane == wlast && c + 4 < LW) right = Ir[c + 4];
            float mo[NDIM][4];
#pragma unroll
            for (int a = 0; a < NDIM; ++a)
#pragma unroll
                for (int j = 0; j < 4; ++j) mo[a][j] = 0.f;
            if (base + tid >= total) return;
            if (y < g.ny && z < g.nz) {
                const float iv[6] = {c > 0 ? left : ic.x, ic.x, ic.y, ic.z, ic.w,
                                     c + 4 < LW ? right : ic.w};
                const float4 yu = lds4(sI + (rI + (y < g.ny - 1 ? 1 : 0)) * LW + c);
                const float4 yd = lds4(sI + (rI - (y > 0 ? 1 : 0)) * LW + c);
                const float yuv[4] = {yu.x, yu.y, yu.z, yu.w}, ydv[4] = {yd.x, yd.y, yd.z, yd.w};
                const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
                float zuv[4] = {0.f, 0.f, 0.f, 0.f}, zdv[4] = {0.f, 0.f, 0.f, 0.f};
                if constexpr (NDIM == 3) {
                    const float4 zu = lds4(sI + (rI + (z < g.nz - 1 ? 6 : 0)) * LW + c);
                    const float4 zd = lds4(sI + (rI - (z > 0 ? 6 : 0)) * LW + c);
                    zuv[0] = zu.x; zuv[1] = zu.y; zuv[2] = zu.z; zuv[3] = zu.w;
                    zdv[0] = zd.x; zdv[1] = zd.y; zdv[2] = zd.z; zdv[3] = zd.w;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int x = x0 - HX + c + j;
                    if (x < 0 || x >= g.nx) continue;
                    const float gx = 0.5f * ((x < g.nx - 1 ? iv[j + 2] : iv[j + 1]) -
                                             (x > 0 ? iv[j] : iv[j + 1]));
                    const float gy = 0.5f * (yuv[j] - ydv[j]);
                    if constexpr (NDIM == 2) {
                        mo[0][j] = pv[j] * gy;
                        mo[1][j] = pv[j] * gx;
                    } else {
                        const float gz = 0.5f * (zuv[j] - zdv[j]);
                        mo[0][j] = pv[j] * gz;
                        mo[1][j] = pv[j] * gy;
                        mo[2][j] = pv[j] * gx;
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < NDIM; ++a)
                *reinterpret_cast<float4*>(sM + (a * kRows + row) * LW + c) =
                    make_float4(mo[a][0], mo[a][1], mo[a][2], mo[a][3]);
        };
        // (pre[]: the first kPre items' p); a warp-uniform trip count: every lane
        // takes part in the shuffles
        int base = 0;
#pragma unroll
        for (int i = 0; i < kPre; ++i, base += kb.ndx())
            if (base < total) form(base, pre[i]);
        for (; base < total; base += kb.ndx()) form(base, load_p(base + tid));
        kb.sync();
        if constexpr (!K::kPersistent) {
            if (s_fail) return;
        }
    }

    // Blur along x: thread (tx, row) -> outputs x0 + 8 tx .. + 7 of `row`,
    // g.txw / 8 threads per row, padded to a multiple of 4 (xpass_threads).
    // Consecutive threads alternate between the two rows of a row pair, so each
    // 8-lane phase of a 16-byte load covers 4 consecutive tx of both rows; with
    // the row stride odd in 16-byte units their 8 addresses fall in the 8
    // distinct bank groups.  The padding lanes only idle here: without them a
    // phase could straddle two row pairs and meet a bank group twice.
    const int tpr = g.txw / kBX, tprp = (tpr + 3) & ~3;
    const int local = tid % (2 * tprp), pair = tid / (2 * tprp);
    const int tx = local >> 1;
    const int row = 2 * pair + (local & 1);
    if (tx >= tpr) return;  // no barrier follows
    const int ty = (NDIM == 2) ? row : (row & 3);
    const int tz = (NDIM == 2) ? 0 : (row >> 2);
    const int y = y0 + ty, z = z0 + tz;
    const int x = x0 + tx * kBX;
    const bool row_ok = (y < g.ny) && (z < g.nz);
    for (int a = 0; a < ncomp; ++a) {
        const float* src = sM + (a * kRows + row) * LW + tx * kBX + (HX - taps.r4);
        float acc[kBX];
#pragma unroll
        for (int j = 0; j < kBX; ++j) acc[j] = 0.f;
        if constexpr (KC > 0) {
            // outputs in pairs (2i, 2i+1) with packed FMAs over even- and
            // odd-aligned input pairs (per lane the scalar fmaf, same order)
            constexpr int NW = 8 * KC + 8;
            float2 ev[NW / 2], od[NW / 2 - 1];
#pragma unroll
            for (int q = 0; q < 2 * KC + 2; ++q) {
                const float4 v = lds4(src + 4 * q);
                ev[2 * q] = make_float2(v.x, v.y);
                ev[2 * q + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int m = 0; m < NW / 2 - 1; ++m) od[m] = make_float2(ev[m].y, ev[m + 1].x);
            float2 a2[kBX / 2];
#pragma unroll
            for (int i = 0; i < kBX / 2; ++i) a2[i] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 8 * KC; ++k) {
                const float2 wt = make_float2(taps.w[k], taps.w[k]);
#pragma unroll
                for (int i = 0; i < kBX / 2; ++i)
                    a2[i] = ffma2(wt, (k & 1) ? od[i + (k >> 1)] : ev[i + (k >> 1)], a2[i]);
            }
#pragma unroll
            for (int i = 0; i < kBX / 2; ++i) {
                acc[2 * i] = a2[i].x;
                acc[2 * i + 1] = a2[i].y;
            }
        } else {
            float4 c0 = lds4(src), c1 = lds4(src + 4);
            for (int kb = 0; kb < taps.kp; kb += 8) {
                const float4 n0 = lds4(src + kb + 8), n1 = lds4(src + kb + 12);
                const float win[16] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w,
                                       n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const float wt = taps.w[kb + kk];
#pragma unroll
                    for (int j = 0; j < kBX; ++j) acc[j] = fmaf(wt, win[j + kk], acc[j]);
                }
                c0 = n0;
                c1 = n1;
            }
        }
        if (row_ok) {
            const int slice = GRADP ? (out_slice0 + a * g.B + b) : (out_slice0 + (int)kb.bz());
            float* o = out + (long long)slice * g.inst + gidx(g, z, y, x);
            if (x < g.P) *reinterpret_cast<float4*>(o) = make_float4(acc[0], acc[1], acc[2], acc[3]);
            if (x + 4 < g.P)
                *reinterpret_cast<float4*>(o + 4) = make_float4(acc[4], acc[5], acc[6], acc[7]);
        }
    }
}


#ifndef META_BODIES_ONLY
template <int NDIM, bool GRADP, int KC>
__global__ void __launch_bounds__(512)
k_xpass(const __grid_constant__ CUtensorMap tmI, const __grid_constant__ CUtensorMap tmP, const __grid_constant__ Taps taps, Geom g, int sliceI, int sliceP, const float* pin, int out_slice0, float* __restrict__ out, unsigned int* fault) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_xpass<HwBlk, NDIM, GRADP, KC>(HwBlk{}, tmI, tmP, taps, g, sliceI, sliceP, pin, out_slice0, out, fault);
}
#endif

// AXIS is the array axis blurred: 2-D: 0 = y; 3-D: 1 = y, 0 = z.
template <class K, int NDIM, int AXIS, int KC>
__device__ __forceinline__ void body_strided(const K& kb, const CUtensorMap& tm, const Taps& taps, Geom g, int in_slice0, int out_slice0, const float* __restrict__ scale, float scale_mul, float* __restrict__ out, unsigned int* fault) {
    unsigned char* smem_raw = kb.smem();
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float* s = reinterpret_cast<float*>(smem_raw + 128);

    const int tid = kb.tx();
    const int pair = tid & 15;           // column pair
    const int grp = tid >> 4;            // group of kBA outputs along the axis
    const int x0 = kb.bx() * kTXS;
    const int slice = kb.bz();           // comp * B + b
    const int b = slice % g.B;
    // tile of L = g.ly or g.lz outputs along the axis, L / kBA warps
    int a0, y, z, n_axis, L;
    if constexpr (NDIM == 2) {
        L = g.ly;
        a0 = kb.by() * L;
        y = 0;
        z = 0;
        n_axis = g.ny;
    } else if constexpr (AXIS == 1) {
        L = g.ly;
        const int nt = (g.ny + L - 1) / L;
        a0 = (kb.by() % nt) * L;
        z = kb.by() / nt;
        y = 0;
        n_axis = g.ny;
    } else {
        L = g.lz;
        const int nt = (g.nz + L - 1) / L;
        a0 = (kb.by() % nt) * L;
        y = kb.by() / nt;
        z = 0;
        n_axis = g.nz;
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    kb.sync();
    if (tid == 0) {
        if constexpr (K::kPersistent) {
            tmap_acquire(&tm);
            fence_proxy_async_global();
        }
        mbar_arrive_expect_tx(bar, (uint32_t)(kTXS * (L + taps.kp) * 4));
        if constexpr (NDIM == 2)
            tma_load_3d(s, &tm, bar, x0, a0 - taps.r, in_slice0 + slice);
        else if constexpr (AXIS == 1)
            tma_load_4d(s, &tm, bar, x0, a0 - taps.r, z, in_slice0 + slice);
        else
            tma_load_4d(s, &tm, bar, x0, y, a0 - taps.r, in_slice0 + slice);
    }
    if constexpr (K::kPersistent) {
        // warp 0 waits (bounded) while the others sleep in the barrier; the tile
        // leaves together if the wait ran out, and the barrier is retired before
        // the next tile reuses the shared memory
        bool landed = true;
        if (tid < 32) landed = mbar_wait_bounded(bar, 0, fault);
        if (kb.sync_or(!landed)) return;
        if (tid == 0) mbar_inval(bar);  // every wait on it has returned
    } else {
        // every warp waits (bounded) itself and starts as soon as the tile has
        // landed: no barrier follows, so a warp whose wait ran out just leaves
        if (!mbar_wait_bounded(bar, 0, fault)) return;
    }

    // Thread (pair, grp): columns x0 + 2 pair and x0 + 2 pair + 1, outputs
    // a0 + 16 grp .. + 15 along the axis.  The two columns form the two lanes of
    // every packed FMA, so tap k reads one aligned 8-byte pair (the inputs of both
    // columns at axis offset j + k) and no pair has to be assembled; each lane is
    // the scalar fmaf chain over the taps in order, as before.
    if (grp >= L / kBA) return;  // lanes that round the CTA up to whole warps
    const float* src = s + (grp * kBA) * kTXS + 2 * pair;
    float2 a2[kBA];
#pragma unroll
    for (int j = 0; j < kBA; ++j) a2[j] = make_float2(0.f, 0.f);
    if constexpr (KC > 0) {
        // taps past 2r are zero padding: their FMAs would add exact zeros, so the
        // last chunk skips them (a uniform test)
        const int khi = 2 * taps.r;
#pragma unroll
        for (int k = 0; k < 8 * KC; ++k) {
            if (k >= 8 * (KC - 1) && k > khi) continue;
            const float2 wt = make_float2(taps.w[k], taps.w[k]);
#pragma unroll
            for (int j = 0; j < kBA; ++j)
                a2[j] = ffma2(wt, lds2(src + (j + k) * kTXS), a2[j]);
        }
    } else {
        for (int kb = 0; kb < taps.kp; kb += 8) {
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const float2 wt = make_float2(taps.w[kb + kk], taps.w[kb + kk]);
#pragma unroll
                for (int j = 0; j < kBA; ++j)
                    a2[j] = ffma2(wt, lds2(src + (j + kb + kk) * kTXS), a2[j]);
            }
        }
    }
    const int x = x0 + 2 * pair;
    if (x >= g.nx) return;
    // outputs a = a0 + grp kBA + j along the axis: one pointer stepped by the
    // axis stride (P for y, slab for z); the pair (x, x + 1) is one 8-byte store
    // (x is even and the row pitch a multiple of 4, so x + 1 < P)
    const int a_first = a0 + grp * kBA;
    const long long stride = (NDIM == 3 && AXIS == 0) ? g.slab : (long long)g.P;
    float* op = out + (long long)(out_slice0 + slice) * g.inst +
                ((NDIM == 2) ? gidx(g, 0, a_first, x)
                             : (AXIS == 1 ? gidx(g, z, a_first, x) : gidx(g, a_first, y, x)));
    const int nj = min(kBA, n_axis - a_first);
    const float sc = scale ? scale_mul * scale[b] : 1.f;
#pragma unroll
    for (int j = 0; j < kBA; ++j) {
        if (j < nj) {
            const float2 v = scale ? make_float2(sc * a2[j].x, sc * a2[j].y) : a2[j];
            *reinterpret_cast<float2*>(op + j * stride) = v;
        }
    }
}


#ifndef META_BODIES_ONLY
template <int NDIM, int AXIS, int KC>
__global__ void __launch_bounds__(256)
k_strided(const __grid_constant__ CUtensorMap tm, const __grid_constant__ Taps taps, Geom g, int in_slice0, int out_slice0, const float* __restrict__ scale, float scale_mul, float* __restrict__ out, unsigned int* fault) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_strided<HwBlk, NDIM, AXIS, KC>(HwBlk{}, tm, taps, g, in_slice0, out_slice0, scale, scale_mul, out, fault);
}
#endif

// Self-test of the failure path: one CTA arms an mbarrier for 16 bytes that no
// copy ever delivers and waits on it exactly as the blur kernels wait on their
// TMA tiles, with a short limit.  The wait runs out, latches kFaultTmaTimeout
// in *fault and the CTA returns; nothing faults and nothing is left in flight.
#ifndef META_BODIES_ONLY
__global__ void __launch_bounds__(64) k_wait_selftest(unsigned int* fault, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) mbar_arrive_expect_tx(&bar, 16u);  // 16 bytes that never arrive
    bool landed = true;
    if (tid < 32) landed = mbar_wait_bounded(&bar, 0, fault, limit_ns);
    if (__syncthreads_or(!landed)) return;
}
#endif

#ifndef META_BODIES_ONLY
cudaError_t launch_wait_selftest(unsigned int* fault, unsigned long long limit_ns, cudaStream_t st) {
    if (recorder()) return cudaErrorNotSupported;  // not replayable by the persistent kernel
    k_wait_selftest<<<1, 64, 0, st>>>(fault, limit_ns);
    return cudaGetLastError();
}

// ------------------------------------------------------------ launchers

size_t xpass_smem(int ndim, bool gradp, int txw, int r, int r4) {
    const int LW = xpass_lw(txw, r, r4);
    if (!gradp) return 128 + (size_t)kRows * LW * 4;
    const int rowsI = ndim == 2 ? kRows + 2 : 36;
    const size_t f = (size_t)((rowsI * LW + 31) & ~31) + (size_t)ndim * kRows * LW;
    return 128 + f * 4;
}

size_t strided_smem(int len, int kp) { return 128 + (size_t)kTXS * (len + kp) * 4; }

template <int NDIM, bool GRADP, int KC>
static cudaError_t launch_xpass_kc(const CUtensorMap& tmI, const CUtensorMap& tmP,
                                   const Taps& taps, const Geom& g, int sliceI, int sliceP,
                                   const float* pin, int out_slice0, int nslices, float* out,
                                   unsigned int* fault, cudaStream_t st) {
    const size_t smem = xpass_smem(NDIM, GRADP, g.txw, taps.r, taps.r4);
    cudaError_t e = cudaFuncSetAttribute(k_xpass<NDIM, GRADP, KC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + g.txw - 1) / g.txw,
              NDIM == 2 ? (g.ny + kRows - 1) / kRows : ((g.ny + 3) / 4) * ((g.nz + 3) / 4),
              GRADP ? g.B : nslices);
    const int threads = xpass_threads(g.txw);
    META_CHECK_LAUNCH(launch_k(k_xpass<NDIM, GRADP, KC>, grid, threads, smem, st, tmI, tmP, taps, g,
                               sliceI, sliceP, pin, out_slice0, out, fault));
    return cudaSuccess;
}

// Compile-time tap loops for up to 7 chunks of 8 (sigma <= 8); runtime beyond.
template <int NDIM, bool GRADP>
static cudaError_t launch_xpass_t(const CUtensorMap& tmI, const CUtensorMap& tmP, const Taps& taps,
                                  const Geom& g, int sliceI, int sliceP, const float* pin, int out_slice0,
                                  int nslices, float* out, unsigned int* fault, cudaStream_t st) {
#define META_XPASS_KC(K)                                                                      \
    case K:                                                                                   \
        return launch_xpass_kc<NDIM, GRADP, K>(tmI, tmP, taps, g, sliceI, sliceP, pin, out_slice0, \
                                               nslices, out, fault, st);
    switch (taps.kp / 8) {
        META_XPASS_KC(1)
        META_XPASS_KC(2)
        META_XPASS_KC(3)
        META_XPASS_KC(4)
        META_XPASS_KC(5)
        META_XPASS_KC(6)
        META_XPASS_KC(7)
        default:
            return launch_xpass_kc<NDIM, GRADP, 0>(tmI, tmP, taps, g, sliceI, sliceP, pin, out_slice0,
                                                   nslices, out, fault, st);
    }
#undef META_XPASS_KC
}

cudaError_t launch_xpass(int ndim, bool gradp, const CUtensorMap& tmI, const CUtensorMap& tmP,
                         const Taps& taps, const Geom& g, int sliceI, int sliceP, const float* pin, int out_slice0,
                         int nslices, float* out, unsigned int* fault, cudaStream_t st) {
    if (std::vector<PRec>* r = recorder()) {
        PRec e{};
        e.kind = PK_XPASS;
        e.ndim = ndim;
        e.sub = gradp ? 1 : 0;
        e.kc = taps.kp / 8;
        e.grid = dim3((g.nx + g.txw - 1) / g.txw,
                      ndim == 2 ? (g.ny + kRows - 1) / kRows : ((g.ny + 3) / 4) * ((g.nz + 3) / 4),
                      gradp ? g.B : nslices);
        e.bx = xpass_threads(g.txw);
        e.by = 1;
        e.smem = xpass_smem(ndim, gradp, g.txw, taps.r, taps.r4);
        e.a.g = g;
        e.a.i0 = sliceI;
        e.a.i1 = sliceP;
        e.a.c[0] = pin;
        e.a.i2 = out_slice0;
        e.a.w[0] = out;
        e.a.fault = fault;
        e.ntm = 2;
        e.tm[0] = tmI;
        e.tm[1] = tmP;
        e.has_taps = 1;
        e.taps = taps;
        r->push_back(e);
        return cudaSuccess;
    }
    if (ndim == 2)
        return gradp ? launch_xpass_t<2, true>(tmI, tmP, taps, g, sliceI, sliceP, pin, out_slice0,
                                               nslices, out, fault, st)
                     : launch_xpass_t<2, false>(tmI, tmP, taps, g, sliceI, sliceP, pin, out_slice0,
                                                nslices, out, fault, st);
    return gradp ? launch_xpass_t<3, true>(tmI, tmP, taps, g, sliceI, sliceP, pin, out_slice0, nslices,
                                           out, fault, st)
                 : launch_xpass_t<3, false>(tmI, tmP, taps, g, sliceI, sliceP, pin, out_slice0,
                                            nslices, out, fault, st);
}

template <int NDIM, int AXIS, int KC>
static cudaError_t launch_strided_kc(const CUtensorMap& tm, const Taps& taps, const Geom& g,
                                     int in_slice0, int out_slice0, int nslices,
                                     const float* scale, float scale_mul, float* out,
                                     unsigned int* fault, cudaStream_t st) {
    const int L = (NDIM == 3 && AXIS == 0) ? g.lz : g.ly;
    const size_t smem = strided_smem(L, taps.kp);
    cudaError_t e = cudaFuncSetAttribute(k_strided<NDIM, AXIS, KC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    unsigned gy;
    if (NDIM == 2)
        gy = (g.ny + L - 1) / L;
    else if (AXIS == 1)
        gy = ((g.ny + L - 1) / L) * g.nz;
    else
        gy = ((g.nz + L - 1) / L) * g.ny;
    dim3 grid((g.nx + kTXS - 1) / kTXS, gy, nslices);
    META_CHECK_LAUNCH(launch_k(k_strided<NDIM, AXIS, KC>, grid, strided_threads(L), smem, st, tm, taps, g,
                               in_slice0, out_slice0, scale, scale_mul, out, fault));
    return cudaSuccess;
}

template <int NDIM, int AXIS>
static cudaError_t launch_strided_t(const CUtensorMap& tm, const Taps& taps, const Geom& g,
                                    int in_slice0, int out_slice0, int nslices,
                                    const float* scale, float scale_mul, float* out,
                                    unsigned int* fault, cudaStream_t st) {
#define META_STRIDED_KC(K)                                                                   \
    case K:                                                                                  \
        return launch_strided_kc<NDIM, AXIS, K>(tm, taps, g, in_slice0, out_slice0, nslices, \
                                                scale, scale_mul, out, fault, st);
    switch (taps.kp / 8) {
        META_STRIDED_KC(1)
        META_STRIDED_KC(2)
        META_STRIDED_KC(3)
        META_STRIDED_KC(4)
        META_STRIDED_KC(5)
        META_STRIDED_KC(6)
        META_STRIDED_KC(7)
        default:
            return launch_strided_kc<NDIM, AXIS, 0>(tm, taps, g, in_slice0, out_slice0, nslices,
                                                    scale, scale_mul, out, fault, st);
    }
#undef META_STRIDED_KC
}

cudaError_t launch_strided(int ndim, int axis, const CUtensorMap& tm, const Taps& taps,
                           const Geom& g, int in_slice0, int out_slice0, int nslices,
                           const float* scale, float scale_mul, float* out, unsigned int* fault,
                           cudaStream_t st) {
    if (std::vector<PRec>* r = recorder()) {
        const int L = (ndim == 3 && axis == 0) ? g.lz : g.ly;
        unsigned gy;
        if (ndim == 2)
            gy = (g.ny + L - 1) / L;
        else if (axis == 1)
            gy = ((g.ny + L - 1) / L) * g.nz;
        else
            gy = ((g.nz + L - 1) / L) * g.ny;
        PRec e{};
        e.kind = PK_STRIDED;
        e.ndim = ndim;
        e.sub = axis;
        e.kc = taps.kp / 8;
        e.grid = dim3((g.nx + kTXS - 1) / kTXS, gy, nslices);
        e.bx = strided_threads(L);
        e.by = 1;
        e.smem = strided_smem(L, taps.kp);
        e.a.g = g;
        e.a.i0 = in_slice0;
        e.a.i1 = out_slice0;
        e.a.c[0] = scale;
        e.a.f0 = scale_mul;
        e.a.w[0] = out;
        e.a.fault = fault;
        e.ntm = 1;
        e.tm[0] = tm;
        e.has_taps = 1;
        e.taps = taps;
        r->push_back(e);
        return cudaSuccess;
    }
    if (ndim == 2)
        return launch_strided_t<2, 0>(tm, taps, g, in_slice0, out_slice0, nslices, scale,
                                      scale_mul, out, fault, st);
    if (axis == 1)
        return launch_strided_t<3, 1>(tm, taps, g, in_slice0, out_slice0, nslices, scale,
                                      scale_mul, out, fault, st);
    return launch_strided_t<3, 0>(tm, taps, g, in_slice0, out_slice0, nslices, scale, scale_mul,
                                  out, fault, st);
}

#endif  // META_BODIES_ONLY

}  // namespace meta
