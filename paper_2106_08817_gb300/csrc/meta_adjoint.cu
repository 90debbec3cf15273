// meta_adjoint.cu -- the cost of Eq. 4 and the discrete adjoint of the
// semi-Lagrangian step (arXiv:2106.08817, Eq. 3-4, Sec. 2.3), sm_103a.
//
// The adjoint runs t = T-1 .. 0 and is the exact transpose of forward step t
// (y = x - dt v, I~ = S(y) I_t, p~ = S(y) p_t, p' = p~ (1 - dt div v),
// I' = I~ + dt mu p~, v = -rho K (p grad I)).  With I^' = I^_{t+1} and
// p^' = p^_{t+1}:
//
//   record of step t at every source x (built by the kernel that produced
//   I^', p^' at x -- the adjoint start k_adj_init from I_T - J or from given
//   gradients, or k_adj_gradp of step t+1):  the cell and f of the foot of x,
//   I^'(x),
//       p~^(x) = p^'(x) (1 - dt div v_t(x)) + dt mu I^'(x),
//       div^(x) = -dt p~_t(x) p^'(x)
//   k_adj_transport2d / 3d  Ihp = S^T I^', php = S^T p~^ (gather over the
//       sources whose foot cell touches the node: fixed order, no atomics) and
//       v^ = -dt y^ + D^T div^, y^ = dI~/dy I^' + dp~/dy p~^ at the node's foot
//   blur of v^ with K = K^T, scaled by -rho (meta_blur.cu)  ->  m^
//   k_adj_gradp2d / k_adj_gradp<3>  p^_t = php + sum_i m^_i D_i I_t,
//                    I^_t = Ihp + sum_i D_i^T (m^_i p_t),
//       then the record of step t-1 (or, at t = 0, the outputs; the cost
//       gradient adds lambda (2 sum_i (D_i I_0)(K m0)_i + 2 rho p0)).
//
// With the det momentum update p' = p~ J, J = det(Id - dt Dv), the record
// holds p~^ = p^' J + dt mu I^' and the same div^, and k_adj_jacT adds the
// part of D^T (div^ cof(Id - dt Dv)) beyond D^T div^ to v^ before the blur.
//
// The Eulerian scheme passes raw adjoints (I^', p^') between steps: k_euler_adj
// transposes its step up to v^, and k_adj_gradp (raw mode) finishes it.  The
// hybrid scheme's image step is semi-Lagrangian: its records (p~^ = dt mu I^',
// div^ = 0) go through the same transport, and k_hybrid_p adds the transpose of
// its Eulerian momentum step.
//
// Each record is built once per voxel, so the transport only gathers.
#include "meta_stencil.cuh"

namespace meta {
namespace {

// Window radius of the gather-form transpose at step t: a source x feeds node
// n only if n lies in the cell of its foot, so |n - x| <= 1 + |d| per axis and
// R = 1 + floor(max |d|) bounds every contributing source.
__device__ __forceinline__ int gather_radius(const unsigned int* maxdisp, int t, int B, int b) {
    return 1 + (int)floorf(__uint_as_float(maxdisp[kMaxdispStride * ((long long)t * B + b)]));
}

// Node tile of the 2-D transport kernel and the largest window gathered;
// beyond it the transport scatters with atomics.
template <int NDIM>
struct GatherTile;
template <>
struct GatherTile<2> {
    static constexpr int TX = 32, TY = 16, RMAX = 8;
};
template <>
struct GatherTile<3> {
    // per-step displacements under 4 voxels: up to 9^3 sources per node, read
    // through L1 in a fixed order (R = 1 marches along z, k_adj_transport3d)
    static constexpr int RMAX = 4;
};

dim3 gather_grid2d(const Geom& g) {
    using G = GatherTile<2>;
    return dim3((g.nx + G::TX - 1) / G::TX, (g.ny + G::TY - 1) / G::TY, g.B);
}

// Foot cell relative to the source: one byte per axis (offset + 64), bit
// 24 + a when the clamp on axis a is inactive.
__device__ __forceinline__ int pack_cell(const int* off, const bool* inside) {
    return (off[0] + 64) | ((off[1] + 64) << 8) | ((off[2] + 64) << 16) |
           (inside[0] ? (1 << 24) : 0) | (inside[1] ? (1 << 25) : 0) |
           (inside[2] ? (1 << 26) : 0);
}
__device__ __forceinline__ int cell_off(int cell, int a) { return ((cell >> (8 * a)) & 0xff) - 64; }

// (D^T w)[c] along a stride s: rows c-1 and c+1 of D, plus the edge rows.
__device__ __forceinline__ float cdiff_T(const float* w, long long o, long long s, int c, int n) {
    float r = 0.f;
    if (c >= 1) r += 0.5f * w[o - s];
    if (c == n - 1) r += 0.5f * w[o];
    if (c <= n - 2) r -= 0.5f * w[o + s];
    if (c == 0) r -= 0.5f * w[o];
    return r;
}

// Record fields: slice (k * B + b) of `rec` for k = 0 cell (int bits),
// 1..NDIM f per axis, NDIM+1 I^', NDIM+2 p~^, NDIM+3 div^.
template <int NDIM>
struct Rec {
    static constexpr int kCell = 0, kI = NDIM + 1, kP = NDIM + 2, kD = NDIM + 3;
};

// The fields of a record (cell bits, f per axis, I^', p~^, div^) in the
// order of Rec.
template <int NDIM>
struct RecVals {
    float v[NDIM + 4];
};

// Record of step t at voxel v from I^' = Ih1, p^' = ph1, the displacement d
// of the foot per axis and fac = div v_t (PDET: fac = J = det(Id - dt Dv_t))
// (the same expressions as the forward step), with p_t at pprev.
template <int NDIM, bool PDET = false, bool HYB = false>
__device__ __forceinline__ RecVals<NDIM> record_values(const Geom& g, const Coefs& cf,
                                                       const Vox& v, float Ih1, float ph1,
                                                       const float* d, float fac,
                                                       const float* pprev) {
    const int b = v.b;
    const float mu = cf.mu[b], dt = cf.dt;
    const Feet<NDIM> F = feet_of<NDIM>(g, v, d);
    float pw = 0.f;
    if constexpr (HYB) {
        // the hybrid's momentum step is Eulerian: p~ is not used and div^ = 0
    } else if constexpr (NDIM == 2) {
        pw = rn_bilin(pprev + F.base, g.P, F.f[0].f, F.f[1].f);
    } else {
        pw = rn_trilin(pprev + F.base, pprev + F.base + g.slab, g.P, F.f[0].f, F.f[1].f,
                       F.f[2].f);
    }
    const int c[3] = {NDIM == 3 ? v.z : v.y, NDIM == 3 ? v.y : v.x, v.x};
    int off[3] = {0, 0, 0};
    bool ins[3] = {false, false, false};
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        off[a] = F.f[a].i0 - c[a];
        ins[a] = F.f[a].inside;
    }
    RecVals<NDIM> r;
    r.v[Rec<NDIM>::kCell] = __int_as_float(pack_cell(off, ins));
#pragma unroll
    for (int a = 0; a < NDIM; ++a) r.v[1 + a] = F.f[a].f;
    r.v[Rec<NDIM>::kI] = Ih1;
    if constexpr (HYB) {
        // I' = I~ + dt mu p~: the adjoint of p~ is dt mu I^'
        r.v[Rec<NDIM>::kP] = __fmul_rn(__fmul_rn(dt, mu), Ih1);
        r.v[Rec<NDIM>::kD] = 0.f;
    } else {
        r.v[Rec<NDIM>::kP] = PDET ? rn_ptilde_hat_J(ph1, Ih1, dt, mu, fac)
                                  : rn_ptilde_hat(ph1, Ih1, dt, mu, fac);
        r.v[Rec<NDIM>::kD] = rn_div_hat(dt, pw, ph1);
    }
    return r;
}

template <int NDIM, bool PDET = false, bool HYB = false>
__device__ __forceinline__ void emit_record(const Geom& g, const Coefs& cf, const Vox& v,
                                            long long o, float Ih1, float ph1, const float* d,
                                            float fac, const float* pprev,
                                            float* rec) {
    const RecVals<NDIM> r = record_values<NDIM, PDET, HYB>(g, cf, v, Ih1, ph1, d, fac, pprev);
    const long long sl = (long long)g.B * g.inst;
    float* w = rec + (long long)v.b * g.inst + o;
#pragma unroll
    for (int k = 0; k < NDIM + 4; ++k) w[k * sl] = r.v[k];
}

// Record of step t at voxel v (pitched offset o in its instance) from
// I^' = Ih1 and p^' = ph1; state t sits in slot s_state, u_t in slot s_u.  The
// same expressions as the forward step t.
template <int NDIM, bool PDET = false, bool HYB = false>
__device__ __forceinline__ void build_record(const Geom& g, const Coefs& cf, int s_state, int s_u,
                                             const Vox& v, long long o, float Ih1, float ph1,
                                             const float* states,
                                             const float* u, float* rec) {
    const int b = v.b;
    const float rho = cf.rho[b], dtrho = cf.dt * rho;
    int c[NDIM], n[NDIM];
    long long s[NDIM];
    axis_info<NDIM>(g, v, c, n, s);
    float d[NDIM];
    float du = 0.f;
    float A[NDIM][NDIM];  // PDET: A[a][e] = D_e u_a
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const float* ua = slice_of(u, g, ((long long)s_u * NDIM + a) * g.B + b);
        d[a] = disp_of(dtrho, ua[o]);
        if constexpr (PDET) {
#pragma unroll
            for (int e = 0; e < NDIM; ++e) {
                const long long hi = (c[e] < n[e] - 1) ? s[e] : 0, lo = (c[e] > 0) ? s[e] : 0;
                A[a][e] = rn_cdiff(ua[o + hi], ua[o - lo]);
            }
        } else {
            const long long hi = (c[a] < n[a] - 1) ? s[a] : 0, lo = (c[a] > 0) ? s[a] : 0;
            du = __fadd_rn(du, rn_cdiff(ua[o + hi], ua[o - lo]));
        }
    }
    const float fac = PDET ? rn_jac_det<NDIM>(A, dtrho) : __fmul_rn(-rho, du);
    emit_record<NDIM, PDET, HYB>(g, cf, v, o, Ih1, ph1, d, fac,
                                 slice_of(states, g, ((long long)s_state * 2 + 1) * g.B + b),
                                 rec);
}

// build_record with the momentum update of the call (cf.pdet), for kernels
// that build records once per call.
template <int NDIM>
__device__ __forceinline__ void build_record_any(const Geom& g, const Coefs& cf, int s_state,
                                                 int s_u, const Vox& v, long long o, float Ih1,
                                                 float ph1, const float* states,
                                                 const float* u, float* rec) {
    if (cf.scheme == 2)
        build_record<NDIM, false, true>(g, cf, s_state, s_u, v, o, Ih1, ph1, states, u, rec);
    else if (cf.pdet)
        build_record<NDIM, true>(g, cf, s_state, s_u, v, o, Ih1, ph1, states, u, rec);
    else
        build_record<NDIM, false>(g, cf, s_state, s_u, v, o, Ih1, ph1, states, u, rec);
}

// The start of the adjoint from the adjoints (Ih1, ph1) of (I_T, p_T): the
// record of step T-1 (semi-Lagrangian, hybrid) and the raw adjoints the
// Eulerian steps read (Eulerian: both; hybrid: ph1 for its momentum step).
template <int NDIM>
__device__ __forceinline__ void adjoint_start(const Geom& g, const Coefs& cf, int s_state,
                                              int s_u, const Vox& v, long long o, float Ih1,
                                              float ph1, const float* states,
                                              const float* u, float* rec,
                                              float* rawI, float* rawP) {
    const long long ob = (long long)v.b * g.inst + o;
    if (cf.scheme != 1)
        build_record_any<NDIM>(g, cf, s_state, s_u, v, o, Ih1, ph1, states, u, rec);
    if (cf.scheme == 1) rawI[ob] = Ih1;
    if (cf.scheme != 0) rawP[ob] = ph1;
}

// Packed per-axis weights of a source whose foot moved by less than one voxel:
// g = f - 1 if its foot cell lies below the source (cell offset -1), g = f
// otherwise.  A source at offset E (-1, 0, +1) from a node passes its value to
// it with weight max(g, 0), 1 - |g|, max(-g, 0) along that axis -- the bilinear
// weights f and 1 - f (1 - |g| = f when the cell lies below holds up to one
// rounding).
__device__ __forceinline__ float pack_g(int off, float f) { return off < 0 ? f - 1.f : f; }
template <int E>
__device__ __forceinline__ float gw(float g) {
    if constexpr (E < 0) return fmaxf(g, 0.f);
    else if constexpr (E > 0) return fmaxf(-g, 0.f);
    else return 1.f - fabsf(g);
}

// ------------------------------------------------------------------ kernels

// Shared memory of the bodies that carve fixed arrays from the block context:
// the cost reductions (3 x 256 doubles), the 2-D transport (8 staged windows of
// 40 x 18 floats and 612 packed float4 sources) and the 2-D gradp (7 staged
// tiles of 40 x 18 floats).
constexpr int kCostSmem = 3 * 256 * 8;
constexpr int kTr2dSmem = (8 * 720 + 4 * 612) * 4;
constexpr int kGradp2dSmem = 7 * (2 * kPY + 2) * (kPX + 8) * 4;

// Cost partials: one CTA = 8 warps over a fixed set of (z, y) rows of
// instance blockIdx.y.  (The adjoint start from I^_T = I_T - J, p^_T = 0 is
// k_adj_init<NDIM, true>, a pointwise kernel of its own.)
template <class K, int NDIM>
__device__ __forceinline__ void body_cost_partials(const K& kb, Geom g, Slots sl, const float* states, const float* u, const float* J, double* partials) {
    const int b = kb.by();
    const long long N = (long long)g.nz * g.ny * g.nx;
    const float* IT = slice_of(states, g, ((long long)sl.sT * 2 + 0) * g.B + b);
    const float* I0 = slice_of(states, g, ((long long)sl.s0 * 2 + 0) * g.B + b);
    const float* p0 = slice_of(states, g, ((long long)sl.s0 * 2 + 1) * g.B + b);
    double data = 0.0, kin = 0.0, res = 0.0;
    // one warp per (z, y) row at a time; a fixed assignment, so fixed sums.
    // Each lane sums its voxels of the row (at most ceil(nx / 32)) in FP32 and
    // adds that to its FP64 totals once per row: FP64 arithmetic runs at a small
    // fraction of the FP32 rate, and per voxel it bound the kernel.
    const int warp = kb.tx() >> 5, lane = kb.tx() & 31;
    const int nrows = g.nz * g.ny;
    for (int row = kb.bx() * 8 + warp; row < nrows; row += kb.gx() * 8) {
        float ds = 0.f, ks = 0.f, rs = 0.f;
        for (int x = lane; x < g.nx; x += 32) {
            Vox v;
            v.b = b;
            v.z = row / g.ny;
            v.y = row - v.z * g.ny;
            v.x = x;
            v.ok = true;
            const long long o = gidx(g, v.z, v.y, v.x);
            const float r = __fsub_rn(IT[o], J[(long long)b * N + (long long)row * g.nx + x]);
            ds = __fmaf_rn(r, r, ds);
            int c[NDIM], n[NDIM];
            long long s[NDIM];
            axis_info<NDIM>(g, v, c, n, s);
            const float p = p0[o];
#pragma unroll
            for (int a = 0; a < NDIM; ++a) {
                const float ga = cdiff(I0, o, s[a], c[a], n[a]);
                const float* ua = slice_of(u, g, ((long long)sl.u0 * NDIM + a) * g.B + b);
                ks = __fmaf_rn(__fmul_rn(p, ga), ua[o], ks);
            }
            rs = __fmaf_rn(p, p, rs);
        }
        data += 0.5 * (double)ds;
        kin += (double)ks;
        res += (double)rs;
    }
    double (*red)[256] = reinterpret_cast<double (*)[256]>(kb.smem());
    red[0][kb.tx()] = data;
    red[1][kb.tx()] = kin;
    red[2][kb.tx()] = res;
    kb.sync();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)kb.tx() < w)
            for (int k = 0; k < 3; ++k) red[k][kb.tx()] += red[k][kb.tx() + w];
        kb.sync();
    }
    if (kb.tx() < 3)
        partials[((long long)b * kb.gx() + kb.bx()) * 3 + kb.tx()] = red[kb.tx()][0];
}


#ifndef META_BODIES_ONLY
template <int NDIM>
__global__ void __launch_bounds__(256)
k_cost_partials(Geom g, Slots sl, const float* __restrict__ states, const float* __restrict__ u, const float* __restrict__ J, double* partials) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_cost_partials<HwBlk, NDIM>(HwBlk{}, g, sl, states, u, J, partials);
}
#endif

template <class K>
__device__ __forceinline__ void body_cost_final(const K& kb, int nblk, Coefs cf, const double* partials, double* cost) {
    const int b = kb.bx();
    double (*red)[256] = reinterpret_cast<double (*)[256]>(kb.smem());
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = kb.tx(); i < nblk; i += kb.ndx())
        for (int k = 0; k < 3; ++k) acc[k] += partials[((long long)b * nblk + i) * 3 + k];
    for (int k = 0; k < 3; ++k) red[k][kb.tx()] = acc[k];
    kb.sync();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)kb.tx() < w)
            for (int k = 0; k < 3; ++k) red[k][kb.tx()] += red[k][kb.tx() + w];
        kb.sync();
    }
    if (kb.tx() == 0) {
        const double lam = (double)cf.lambda[b], rho = (double)cf.rho[b];
        cost[b * 3 + 0] = red[0][0];
        cost[b * 3 + 1] = lam * red[1][0];
        cost[b * 3 + 2] = lam * rho * red[2][0];
    }
}


#ifndef META_BODIES_ONLY
__global__ void __launch_bounds__(256)
k_cost_final(int nblk, Coefs cf, const double* __restrict__ partials, double* cost) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_cost_final<HwBlk>(HwBlk{}, nblk, cf, partials, cost);
}
#endif

// Adjoint start from given gradients w.r.t. (I_T, p_T): record of step T-1
// (and the raw adjoints of the Eulerian steps).  FROM_J: the cost's start,
// I^_T = I_T - J with J (contiguous) in gI1, p^_T = 0.
template <class K, int NDIM, bool FROM_J>
__device__ __forceinline__ void body_adj_init(const K& kb, Geom g, Coefs cf, Slots sl, const float* states, const float* u, const float* gI1, const float* gp1, const unsigned int* maxdisp, float* rec, float* Ihp, float* php, float* rawI, float* rawP) {
    const Vox v = vox_of<NDIM>(g, kb);
    if (!v.ok) return;
    const long long o = gidx(g, v.z, v.y, v.x);
    const long long ci = cidx(g, v);
    float Ih1, ph1 = 0.f;
    if constexpr (FROM_J) {
        Ih1 = slice_of(states, g, ((long long)sl.sT * 2 + 0) * g.B + v.b)[o] - gI1[ci];
    } else {
        Ih1 = gI1[ci];
        ph1 = gp1 ? gp1[ci] : 0.f;
    }
    adjoint_start<NDIM>(g, cf, sl.st1, sl.ut1, v, o, Ih1, ph1, states, u, rec, rawI, rawP);
    if (gather_radius(maxdisp, g.nT - 1, g.B, v.b) > GatherTile<NDIM>::RMAX) {
        slice_of(Ihp, g, v.b)[o] = 0.f;  // the first transport scatters into these
        slice_of(php, g, v.b)[o] = 0.f;
    }
}


#ifndef META_BODIES_ONLY
template <int NDIM, bool FROM_J>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_init(Geom g, Coefs cf, Slots sl, const float* __restrict__ states, const float* __restrict__ u, const float* __restrict__ gI1, const float* __restrict__ gp1, const unsigned int* __restrict__ maxdisp, float* rec, float* Ihp, float* php, float* rawI, float* rawP) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_adj_init<HwBlk, NDIM, FROM_J>(HwBlk{}, g, cf, sl, states, u, gI1, gp1, maxdisp, rec, Ihp, php, rawI, rawP);
}
#endif

// 2-D adjoint step t with R = 1 on a 32 x 16 tile (two rows per thread), all
// operands staged: the records (cell, f_y, f_x, I^', p~^, div^) and I_t, p_t
// over the tile grown by one voxel, by cp.async.  Each source of the grown tile is packed once into the float4
// (g_y, g_x, I^', p~^) (pack_g); each node then sums 9 branch-free products.
template <class K>
__device__ __forceinline__ void transport_r1_2d(const K& kb, const Geom& g, float dt, const float* rb,
                                                long long sl, const float* It, const float* pt,
                                                float* vh0, float* vh1, float* Ihpb,
                                                float* phpb, float* smem) {
    constexpr int TX = 32, TY = 16, W = TX + 8, HR = TY + 2, WIN = W * HR;
    constexpr int RX = TX + 2, RY = TY + 2, NR = RX * RY;
    const int x0 = kb.bx() * TX, y0 = kb.by() * TY;
    const int tx = kb.tx(), ty = kb.ty(), tid = ty * kPX + tx;
    float* sC = smem;            // cell bits
    float* sF0 = sC + WIN;
    float* sF1 = sF0 + WIN;
    float* sI = sF1 + WIN;       // I^'
    float* sP = sI + WIN;        // p~^
    float* sD = sP + WIN;        // div^
    float* sIt = sD + WIN;
    float* sPt = sIt + WIN;
    float4* sQ = reinterpret_cast<float4*>(sPt + WIN);  // [NR]: g_y, g_x, I^', p~^
    const int xl = x0 - 4, yl = y0 - 1;
    stage_async<W, HR>(sC, rb, g, xl, yl, tid);
    stage_async<W, HR>(sF0, rb + sl, g, xl, yl, tid);
    stage_async<W, HR>(sF1, rb + 2 * sl, g, xl, yl, tid);
    stage_async<W, HR>(sI, rb + 3 * sl, g, xl, yl, tid);
    stage_async<W, HR>(sP, rb + 4 * sl, g, xl, yl, tid);
    stage_async<W, HR>(sD, rb + 5 * sl, g, xl, yl, tid);
    stage_async<W, HR>(sIt, It, g, xl, yl, tid);
    stage_async<W, HR>(sPt, pt, g, xl, yl, tid);
    cp_async_wait_all();
    kb.sync();
    for (int i = tid; i < NR; i += kPX * kPY) {
        const int ry = i / RX, rx = i - ry * RX;
        const int sx = x0 - 1 + rx, sy = y0 - 1 + ry;
        const int wi = ry * W + rx + 3;  // window index of source (sy, sx)
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);  // outside: no weight, no value
        if (sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny) {
            const int cell = __float_as_int(sC[wi]);
            q = make_float4(pack_g(cell_off(cell, 0), sF0[wi]), pack_g(cell_off(cell, 1), sF1[wi]),
                            sI[wi], sP[wi]);
        }
        sQ[i] = q;
    }
    kb.sync();
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {  // rows ty and ty + 8 of the tile
        const int ly = ty + rr * kPY;
        const int x = x0 + tx, y = y0 + ly;
        if (x >= g.nx || y >= g.ny) continue;
        const int me = (ly + 1) * RX + tx + 1;  // region index of the node
        const int mw = (ly + 1) * W + tx + 4;   // window index of the node
        float2 acc = make_float2(0.f, 0.f);     // S^T I^', S^T p~^ (one packed FMA per source)
        // the source at offset (dy, dx) from the node passes weight gw<dy> gw<dx>
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const float4 q = sQ[me + dy * RX + dx];
                float wy, wx;
                if (dy < 0) wy = gw<-1>(q.x); else if (dy > 0) wy = gw<1>(q.x); else wy = gw<0>(q.x);
                if (dx < 0) wx = gw<-1>(q.y); else if (dx > 0) wx = gw<1>(q.y); else wx = gw<0>(q.y);
                const float wgt = wy * wx;
                acc = ffma2(make_float2(wgt, wgt), make_float2(q.z, q.w), acc);
            }
        }
        const int o = y * g.P + x;
        Ihpb[o] = acc.x;
        phpb[o] = acc.y;
        // y^ from the node's own foot (cell within one voxel of the node)
        const int cell = __float_as_int(sC[mw]);
        const float fy = sF0[mw], fx = sF1[mw];
        const bool iny = (cell >> 24) & 1, inx = (cell >> 25) & 1;
        // (R = 1: the cell is the node's own or the one below on each axis)
        const int ci = mw + chk_range(g, cell_off(cell, 0), -1, 0) * W +
                       chk_range(g, cell_off(cell, 1), -1, 0);
        float dIy, dIx, dPy, dPx;
        bilin_grad(sIt + ci, W, fy, fx, iny, inx, &dIy, &dIx);
        bilin_grad(sPt + ci, W, fy, fx, iny, inx, &dPy, &dPx);
        const float Ihv = sI[mw], pthv = sP[mw];
        float dT0 = 0.f, dT1 = 0.f;
        if (y >= 1) dT0 += 0.5f * sD[mw - W];
        if (y == g.ny - 1) dT0 += 0.5f * sD[mw];
        if (y <= g.ny - 2) dT0 -= 0.5f * sD[mw + W];
        if (y == 0) dT0 -= 0.5f * sD[mw];
        if (x >= 1) dT1 += 0.5f * sD[mw - 1];
        if (x == g.nx - 1) dT1 += 0.5f * sD[mw];
        if (x <= g.nx - 2) dT1 -= 0.5f * sD[mw + 1];
        if (x == 0) dT1 -= 0.5f * sD[mw];
        vh0[o] = -dt * (dIy * Ihv + dPy * pthv) + dT0;
        vh1[o] = -dt * (dIx * Ihv + dPx * pthv) + dT1;
    }
}

// Records of step t from raw adjoints I^_{t+1}, p^_{t+1} (pitched), once the
// forward segment holding step t has been recomputed (step checkpointing).
template <class K, int NDIM>
__device__ __forceinline__ void body_adj_records(const K& kb, Geom g, Coefs cf, Slots sl, const float* states, const float* u, const float* rawI, const float* rawP, float* rec) {
    const Vox v = vox_of<NDIM>(g, kb);
    if (!v.ok) return;
    const long long o = gidx(g, v.z, v.y, v.x);
    const long long ob = (long long)v.b * g.inst + o;
    build_record_any<NDIM>(g, cf, sl.st1, sl.ut1, v, o, rawI[ob], rawP[ob], states, u, rec);
}


#ifndef META_BODIES_ONLY
template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_records(Geom g, Coefs cf, Slots sl, const float* __restrict__ states, const float* __restrict__ u, const float* __restrict__ rawI, const float* __restrict__ rawP, float* rec) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_adj_records<HwBlk, NDIM>(HwBlk{}, g, cf, sl, states, u, rawI, rawP, rec);
}
#endif

// S^T and v^ of adjoint step t at one node v, from the records of step t in
// global memory, for R > 1 (R = 1 has staged paths below).
//   1 < R <= RMAX: the node gathers over its (2R+1)^d window in a fixed order.
//   R > RMAX: the node's own source scatters its 2^d corner terms with
//     atomics into the zeroed Ihp / php (bounded work; summation order not
//     fixed; info bit).
template <int NDIM, class K>
__device__ __forceinline__ void transport_node(const K& kb, const Geom& g, const Coefs& cf,
                                               const Slots& sl,
                                               const float* states, int R,
                                               const float* rec, float* vh,
                                               float* Ihp, float* php, unsigned int* fault,
                                               const Vox& v) {
    const int b = v.b;
    const long long rsl = (long long)g.B * g.inst;
    const float* rb = rec + (long long)b * g.inst;  // record field k at rb + k * rsl
    const float* rI = rb + Rec<NDIM>::kI * rsl;
    const float* rP = rb + Rec<NDIM>::kP * rsl;
    const float* rD = rb + Rec<NDIM>::kD * rsl;
    const long long o = gidx(g, v.z, v.y, v.x);
    int c[NDIM], n[NDIM];
    long long st[NDIM];
    axis_info<NDIM>(g, v, c, n, st);
    if (R <= GatherTile<NDIM>::RMAX) {
        float accI = 0.f, accP = 0.f;
        int lo[NDIM], hi[NDIM];
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            lo[a] = max(c[a] - R, 0);
            hi[a] = min(c[a] + R, n[a] - 1);
        }
        int e[3];
        const int zlo = (NDIM == 3) ? lo[0] : 0, zhi = (NDIM == 3) ? hi[0] : 0;
        for (int sz = zlo; sz <= zhi; ++sz) {
            for (int sy = lo[NDIM - 2]; sy <= hi[NDIM - 2]; ++sy) {
                for (int sx = lo[NDIM - 1]; sx <= hi[NDIM - 1]; ++sx) {
                    const long long so = gidx(g, sz, sy, sx);
                    const int cell = __float_as_int(ld_ro<K>(rb + so));
                    const int sc[3] = {NDIM == 3 ? sz : sy, NDIM == 3 ? sy : sx, sx};
                    bool hit = true;
#pragma unroll
                    for (int a = 0; a < NDIM; ++a) {
                        e[a] = c[a] - sc[a] - cell_off(cell, a);  // node - foot cell: 0 or 1
                        hit = hit && (unsigned)e[a] <= 1u;
                    }
                    if (!hit) continue;
                    float w = 1.f;
#pragma unroll
                    for (int a = 0; a < NDIM; ++a) {
                        const float f = ld_ro<K>(rb + (1 + a) * rsl + so);
                        w = (a == 0) ? (e[a] ? f : 1.f - f) : w * (e[a] ? f : 1.f - f);
                    }
                    accI += w * ld_ro<K>(rI + so);
                    accP += w * ld_ro<K>(rP + so);
                }
            }
        }
        Ihp[(long long)b * g.inst + o] = accI;
        php[(long long)b * g.inst + o] = accP;
    } else {
        if (kb.tx() == 0 && kb.ty() == 0) atomicOr(fault, kInfoScatter);
        const int cell = __float_as_int(ld_ro<K>(rb + o));
        const float fI = ld_ro<K>(rI + o), fP = ld_ro<K>(rP + o);
        float f[NDIM];
        long long q0 = 0;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            f[a] = ld_ro<K>(rb + (1 + a) * rsl + o);
            q0 += (long long)chk_range(g, c[a] + cell_off(cell, a), 0, n[a] - 2) * st[a];
        }
        float* Isc = Ihp + (long long)b * g.inst;
        float* Psc = php + (long long)b * g.inst;
#pragma unroll
        for (int k = 0; k < (1 << NDIM); ++k) {
            float w = 1.f;
            long long q = q0;
#pragma unroll
            for (int a = 0; a < NDIM; ++a) {
                const int up = (k >> a) & 1;
                w *= up ? f[a] : 1.f - f[a];
                q += up ? st[a] : 0;
            }
            atomicAdd(Isc + q, w * fI);
            atomicAdd(Psc + q, w * fP);
        }
    }

    // y^ from this node's own foot, v^ = -dt y^ + D^T div^.
    const float dt = cf.dt;
    const int cell = __float_as_int(ld_ro<K>(rb + o));
    Feet<NDIM> F;
    int i0[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        i0[a] = chk_range(g, c[a] + cell_off(cell, a), 0, n[a] - 2);
        F.f[a].i0 = i0[a];
        F.f[a].f = ld_ro<K>(rb + (1 + a) * rsl + o);
        F.f[a].inside = (cell >> (24 + a)) & 1;
    }
    if constexpr (NDIM == 2)
        F.base = gidx(g, 0, i0[0], i0[1]);
    else
        F.base = gidx(g, i0[0], i0[1], i0[2]);
    const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
    float Iv, pv, dI[NDIM], dP[NDIM];
    interp_grad<NDIM>(g, F, It, &Iv, dI);
    interp_grad<NDIM>(g, F, pt, &pv, dP);
    const float Ihv = ld_ro<K>(rI + o), pthv = ld_ro<K>(rP + o);
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const float yh = dI[a] * Ihv + dP[a] * pthv;
        vh[((long long)a * g.B + b) * g.inst + o] = -dt * yh + cdiff_T(rD, o, st[a], c[a], n[a]);
    }
}

// 2-D S^T and v^ of adjoint step t: transport_r1_2d when every per-step
// displacement is under one voxel (R = 1), else transport_node per node.
template <class K>
__device__ __forceinline__ void body_adj_transport2d(const K& kb, Geom g, Coefs cf, int t, Slots sl, const float* states, const unsigned int* maxdisp, const float* rec, float* vh, float* Ihp, float* php, unsigned int* fault) {
    // 8 staged windows of 40 x 18 and 34 x 18 packed sources (transport_r1_2d)
    float* s2 = reinterpret_cast<float*>(kb.smem());
    using G = GatherTile<2>;
    const int b = kb.bz();
    const int R = gather_radius(maxdisp, t, g.B, b);
    if (R == 1) {  // uniform over the CTA
        const long long rsl = (long long)g.B * g.inst;
        transport_r1_2d(kb, g, cf.dt, rec + (long long)b * g.inst, rsl,
                        slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b),
                        slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b),
                        vh + (long long)b * g.inst, vh + ((long long)g.B + b) * g.inst,
                        Ihp + (long long)b * g.inst, php + (long long)b * g.inst, s2);
        return;
    }
    for (int rr = 0; rr < 2; ++rr) {
        Vox v;
        v.b = b;
        v.x = kb.bx() * G::TX + kb.tx();
        v.y = kb.by() * G::TY + kb.ty() + rr * kPY;
        v.z = 0;
        if (v.x >= g.nx || v.y >= g.ny) continue;
        transport_node<2>(kb, g, cf, sl, states, R, rec, vh, Ihp, php, fault, v);
    }
}


#ifndef META_BODIES_ONLY
__global__ void __launch_bounds__(kPX * kPY)
k_adj_transport2d(Geom g, Coefs cf, int t, Slots sl, const float* __restrict__ states, const unsigned int* __restrict__ maxdisp, const float* __restrict__ rec, float* vh, float* Ihp, float* php, unsigned int* fault) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_adj_transport2d<HwBlk>(HwBlk{}, g, cf, t, sl, states, maxdisp, rec, vh, Ihp, php, fault);
}
#endif

// 3-D S^T and v^ of adjoint step t.  A CTA owns a 32 x kTransRows (8) column of nodes
// over planes [zs, zs + zc) and marches along z; each thread owns the two
// adjacent nodes (x, 2 ty) and (x, 2 ty + 1) of the column.
//   R = 1: plane p of the records and of I_t, p_t over the column grown by one
//     voxel in x and y is staged by TMA (three bulk tensor copies issued by
//     one thread, completion on an mbarrier per plane parity, plane p + 1 in
//     flight while plane p is used) into two rings: the record fields used
//     only when the plane is packed and when its own nodes complete (cell,
//     f_z, f_y, f_x, I^', p~^; 3 slots) and the fields read from the planes
//     around a completing node (div^, I_t, p_t; 4 slots).  The sources of the
//     plane are packed once into the float4 (g_z, g_y, g_x, I^') and p~^,
//     where per axis g = f - 1 if the foot cell lies below the source (cell
//     offset -1) and g = f otherwise.  The weight with which a source at
//     offset e from a node passes its value along one axis is then max(g, 0)
//     for e = -1, 1 - |g| for e = 0, max(-g, 0) for e = +1 (the bilinear
//     weights f and 1 - f; 1 - |g| = f when the cell lies below holds up to
//     one rounding).  Each thread reads the 12 sources of plane p around its
//     two nodes once (rows 2 ty - 1 .. 2 ty + 2: the middle two serve both
//     nodes) and adds them, in the order (row, column) of each node's 3 x 3
//     window, to the running sums of its nodes at planes p+1, p, p-1
//     (branch-free; zero weights add exact zeros); the nodes at p-1 are then
//     complete and take y^, D^T div^ from the staged planes p-2 .. p.
//   R > 1: transport_node for each node of the column.
constexpr int kMTY = kTransRows / 2;                     // threads along y (two rows each)
constexpr int kMThreads = kPX * kMTY;
constexpr int kMW = 40, kMHY = kTransRows + 2, kMPL = kMW * kMHY;  // staged window (x, y) of a plane
constexpr int kMRX = 34, kMRY = kTransRows + 2, kMPR = kMRX * kMRY;  // source region of a plane
constexpr int kMFA = 6;                                  // ring A: cell f_z f_y f_x I^' p~^
constexpr int kMSA = kMFA * kMPL;                        // ring A slot (floats)
constexpr int kMBI = (kMPL + 31) / 32 * 32, kMBP = kMBI + kMPL;  // ring B: div^ at 0, I_t, p_t
constexpr int kMSB = kMBP + kMPL;                        // ring B slot (floats, 128-byte multiple)
constexpr int kMSlotsA = 3, kMSlotsB = 4;
constexpr size_t kMarchSmem =
    128 + (size_t)(kMSlotsA * kMSA + kMSlotsB * kMSB + 5 * kMPR) * sizeof(float);
constexpr uint32_t kMBytesA = kMFA * kMPL * 4, kMBytesB = 3 * kMPL * 4;
static_assert((kMSA * 4) % 128 == 0 && (kMSB * 4) % 128 == 0 && (kMBI * 4) % 128 == 0,
              "TMA destinations start on 128-byte boundaries");

// Packs the sources of one staged plane at z (zero outside the domain) from
// its ring-A slot.
__device__ __forceinline__ void march_pack(const float* raw, float4* q, float* pp, const Geom& g,
                                           int x0, int y0, int z, int tid) {
    const bool zin = z >= 0 && z < g.nz;
    for (int i = tid; i < kMPR; i += kMThreads) {
        const int ry = i / kMRX, rx = i - ry * kMRX;
        const int sx = x0 - 1 + rx, sy = y0 - 1 + ry;
        const int wi = ry * kMW + rx + 3;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        float pv = 0.f;
        if (zin && sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny) {
            const int cell = __float_as_int(raw[wi]);
            const float fz = raw[kMPL + wi], fy = raw[2 * kMPL + wi], fx = raw[3 * kMPL + wi];
            v.x = pack_g(cell_off(cell, 0), fz);
            v.y = pack_g(cell_off(cell, 1), fy);
            v.z = pack_g(cell_off(cell, 2), fx);
            v.w = raw[4 * kMPL + wi];
            pv = raw[5 * kMPL + wi];
        }
        q[i] = v;
        pp[i] = pv;
    }
}

// Weight of a source at offset E from a node along one axis, from its packed g.
template <int E>
__device__ __forceinline__ float gwe(float g) {
    if constexpr (E < 0) return gw<-1>(g);
    else if constexpr (E > 0) return gw<1>(g);
    else return gw<0>(g);
}

// Adds the packed source (qv, pv) at offset (DY, DX) in y and x of a node to
// its running sums at the planes below, at and above the source's plane,
// with the z weights zm, z0, zp of the source.
template <int DY, int DX>
__device__ __forceinline__ void gather_add(const float4& qv, float pv, float wx, float zm, float z0,
                                           float zp, float2& am, float2& a0, float2& ap) {
    const float wyx = gwe<DY>(qv.y) * wx;
    const float2 tv = fmul2(make_float2(wyx, wyx), make_float2(qv.w, pv));
    am = ffma2(make_float2(zm, zm), tv, am);
    a0 = ffma2(make_float2(z0, z0), tv, a0);
    ap = ffma2(make_float2(zp, zp), tv, ap);
}

// y^ and D^T div^ of the completed node (z, y, x) (window index mw in its
// plane), and its outputs.
__device__ __forceinline__ void transport_complete(const Geom& g, float dt, int b, int z, int y,
                                                   int x, int mw, const float* A_z,
                                                   const float* B_zm, const float* B_z,
                                                   const float* B_zp, const float* B_lo,
                                                   const float* B_hi, float2 acc, float* vh,
                                                   float* Ihp, float* php) {
    const long long o = gidx(g, z, y, x);
    Ihp[(long long)b * g.inst + o] = acc.x;
    php[(long long)b * g.inst + o] = acc.y;
    const int cell = __float_as_int(A_z[mw]);
    const float fz = A_z[kMPL + mw], fy = A_z[2 * kMPL + mw], fx = A_z[3 * kMPL + mw];
    // (R = 1: the cell is the node's own or the one below on each axis)
    const int ci = mw + chk_range(g, cell_off(cell, 1), -1, 0) * kMW +
                   chk_range(g, cell_off(cell, 2), -1, 0);
    const bool inz = (cell >> 24) & 1, iny = (cell >> 25) & 1, inx = (cell >> 26) & 1;
    float Iv, pv, dI[3], dP[3];
    trilin_grad_pq(B_lo + kMBI + ci, B_hi + kMBI + ci, kMW, fz, fy, fx, inz, iny, inx, &Iv, dI);
    trilin_grad_pq(B_lo + kMBP + ci, B_hi + kMBP + ci, kMW, fz, fy, fx, inz, iny, inx, &pv, dP);
    const float Ihv = A_z[4 * kMPL + mw], pthv = A_z[5 * kMPL + mw];
    float dT[3];
    {  // (D^T div^) along z: the neighbouring planes' div^
        float r = 0.f;
        if (z >= 1) r += 0.5f * B_zm[mw];
        if (z == g.nz - 1) r += 0.5f * B_z[mw];
        if (z <= g.nz - 2) r -= 0.5f * B_zp[mw];
        if (z == 0) r -= 0.5f * B_z[mw];
        dT[0] = r;
    }
    const int c2[2] = {y, x}, n2[2] = {g.ny, g.nx}, s2[2] = {kMW, 1};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        float r = 0.f;
        if (c2[a] >= 1) r += 0.5f * B_z[mw - s2[a]];
        if (c2[a] == n2[a] - 1) r += 0.5f * B_z[mw];
        if (c2[a] <= n2[a] - 2) r -= 0.5f * B_z[mw + s2[a]];
        if (c2[a] == 0) r -= 0.5f * B_z[mw];
        dT[1 + a] = r;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        vh[((long long)a * g.B + b) * g.inst + o] = -dt * (dI[a] * Ihv + dP[a] * pthv) + dT[a];
}

template <class K>
__device__ __forceinline__ void body_adj_transport3d(const K& kb, const CUtensorMap& tmRecA, const CUtensorMap& tmRecD, const CUtensorMap& tmSt, Geom g, Coefs cf, int t, Slots sl, int zc, const float* states, const unsigned int* maxdisp, const float* rec, float* vh, float* Ihp, float* php, unsigned int* fault) {
    unsigned char* smem_raw = kb.smem();
    const int b = kb.bz();
    const int nxc = (g.nx + 31) / 32;
    const int x0 = (kb.bx() % nxc) * 32;
    const int zs = (kb.bx() / nxc) * zc;
    const int ze = min(zs + zc, g.nz);
    const int y0 = kb.by() * kTransRows;
    const int R = gather_radius(maxdisp, t, g.B, b);
    const int tx = kb.tx(), ty = kb.ty();
    const int tid = ty * kPX + tx;
    const int x = x0 + tx, ya = y0 + 2 * ty, yb = ya + 1;
    const bool ok_a = x < g.nx && ya < g.ny, ok_b = x < g.nx && yb < g.ny;
    if (R != 1) {  // uniform over the CTA
        Vox v;
        v.b = b;
        v.x = x;
        for (int z = zs; z < ze; ++z) {
            v.z = z;
            v.y = ya;
            if (ok_a) transport_node<3>(kb, g, cf, sl, states, R, rec, vh, Ihp, php, fault, v);
            v.y = yb;
            if (ok_b) transport_node<3>(kb, g, cf, sl, states, R, rec, vh, Ihp, php, fault, v);
        }
        return;
    }
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // [2]: planes of even / odd index
    float* ringA = reinterpret_cast<float*>(smem_raw + 128);
    float* ringB = ringA + kMSlotsA * kMSA;
    float4* Q = reinterpret_cast<float4*>(ringB + kMSlotsB * kMSB);  // [kMPR]
    float* PP = reinterpret_cast<float*>(Q + kMPR);                  // [kMPR]
    // plane p sits in slots (p - zs + 1) mod 3 of A and mod 4 of B
    auto slotA = [&](int p) { return ringA + ((p - zs + 1) % kMSlotsA) * kMSA; };
    auto slotB = [&](int p) { return ringB + ((p - zs + 1) & 3) * kMSB; };
    // every warp waits (bounded) for each plane itself; a wait that runs out raises
    // s_fail, which all threads read after the barrier that follows the packing
    __shared__ int s_fail;
    if (tid == 0) {
        s_fail = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        if constexpr (K::kPersistent) {
            tmap_acquire(&tmRecA);
            tmap_acquire(&tmRecD);
            tmap_acquire(&tmSt);
            fence_proxy_async_global();
        }
    }
    kb.sync();
    // one thread stages plane p: records 0..5 into A, div^ and (I_t, p_t) into
    // B; planes outside the volume are never read, so no copy is made for them
    auto load_plane = [&](int p) {
        uint64_t* br = &bar[(p - zs + 1) & 1];
        if (p >= 0 && p < g.nz) {
            mbar_arrive_expect_tx(br, kMBytesA + kMBytesB);
            float* dB = slotB(p);
            tma_load_5d(slotA(p), &tmRecA, br, x0 - 4, y0 - 1, p, b, 0);
            tma_load_5d(dB, &tmRecD, br, x0 - 4, y0 - 1, p, b, Rec<3>::kD);
            tma_load_5d(dB + kMBI, &tmSt, br, x0 - 4, y0 - 1, p, b, 2 * sl.st);
        } else {
            mbar_arrive(br);
        }
    };
    const float dt = cf.dt;
    const int mwa = (2 * ty + 1) * kMW + tx + 4;   // window index of node a in a plane
    const int mea = (2 * ty + 1) * kMRX + tx + 1;  // region index of node a in a plane
    // running sums (S^T I^', S^T p~^) of both nodes at planes p-1, p, p+1
    float2 am_a = make_float2(0.f, 0.f), a0_a = am_a, ap_a = am_a;
    float2 am_b = am_a, a0_b = am_a, ap_b = am_a;
    if (tid == 0) load_plane(zs - 1);
    for (int p = zs - 1; p <= ze; ++p) {
        const int j = p - zs + 1;  // planes staged so far
        kb.sync();  // every read of the slots plane p + 1 reuses, and of Q / PP, is done
        if (tid == 0 && p + 1 <= ze) load_plane(p + 1);
        if (!mbar_wait_bounded(&bar[j & 1], (j >> 1) & 1, fault)) s_fail = 1;
        // (after a wait ran out the packing reads stale words at fixed in-bounds
        // indices; its results are dropped below)
        march_pack(slotA(p), Q, PP, g, x0, y0, p, tid);
        kb.sync();
        if (s_fail) {
            // leave together, after the copy of plane p + 1 (if any) has landed
            if (tid < 32 && p + 1 <= ze)
                mbar_wait_bounded(&bar[(j + 1) & 1], ((j + 1) >> 1) & 1, fault, 100000000ull);
            kb.sync();
            return;
        }
        // plane p is at dz = -1 from nodes at p+1, 0 from p, +1 from p-1.  Sources
        // r = 0..3 (rows 2 ty - 1 .. 2 ty + 2 of the column), columns dx = 0..2
        // (x - 1 .. x + 1), each loaded and weighted along x and z once; each
        // node adds its nine in its own order: rows dy = -1, 0, 1 outer, columns
        // inner
#define META_SRC(r, dx)                                                                   \
        const float4 q##r##_##dx = Q[mea + (r - 1) * kMRX + (dx - 1)];                    \
        const float p##r##_##dx = PP[mea + (r - 1) * kMRX + (dx - 1)];                    \
        const float wx##r##_##dx = gwe<dx - 1>(q##r##_##dx.z);                            \
        const float zm##r##_##dx = gw<1>(q##r##_##dx.x), z0##r##_##dx = gw<0>(q##r##_##dx.x), \
                    zp##r##_##dx = gw<-1>(q##r##_##dx.x);
        META_SRC(0, 0) META_SRC(0, 1) META_SRC(0, 2)
        META_SRC(1, 0) META_SRC(1, 1) META_SRC(1, 2)
        META_SRC(2, 0) META_SRC(2, 1) META_SRC(2, 2)
        META_SRC(3, 0) META_SRC(3, 1) META_SRC(3, 2)
#undef META_SRC
#define META_ADD(r, dx, DY, am, a0, ap)                                                   \
        gather_add<DY, dx - 1>(q##r##_##dx, p##r##_##dx, wx##r##_##dx, zm##r##_##dx,      \
                               z0##r##_##dx, zp##r##_##dx, am, a0, ap);
        // node a: source rows 0, 1, 2 at dy = -1, 0, 1
        META_ADD(0, 0, -1, am_a, a0_a, ap_a) META_ADD(0, 1, -1, am_a, a0_a, ap_a)
        META_ADD(0, 2, -1, am_a, a0_a, ap_a)
        META_ADD(1, 0, 0, am_a, a0_a, ap_a) META_ADD(1, 1, 0, am_a, a0_a, ap_a)
        META_ADD(1, 2, 0, am_a, a0_a, ap_a)
        META_ADD(2, 0, 1, am_a, a0_a, ap_a) META_ADD(2, 1, 1, am_a, a0_a, ap_a)
        META_ADD(2, 2, 1, am_a, a0_a, ap_a)
        // node b: source rows 1, 2, 3 at dy = -1, 0, 1
        META_ADD(1, 0, -1, am_b, a0_b, ap_b) META_ADD(1, 1, -1, am_b, a0_b, ap_b)
        META_ADD(1, 2, -1, am_b, a0_b, ap_b)
        META_ADD(2, 0, 0, am_b, a0_b, ap_b) META_ADD(2, 1, 0, am_b, a0_b, ap_b)
        META_ADD(2, 2, 0, am_b, a0_b, ap_b)
        META_ADD(3, 0, 1, am_b, a0_b, ap_b) META_ADD(3, 1, 1, am_b, a0_b, ap_b)
        META_ADD(3, 2, 1, am_b, a0_b, ap_b)
#undef META_ADD
        const int z = p - 1;  // complete: planes z-1 .. z+1 added
        if (z >= zs) {
            const float* A_z = slotA(z);
            const float *B_zm = slotB(z - 1), *B_z = slotB(z), *B_zp = slotB(z + 1);
            if (ok_a) {
                const int oz = cell_off(__float_as_int(A_z[mwa]), 0);
                transport_complete(g, dt, b, z, ya, x, mwa, A_z, B_zm, B_z, B_zp,
                                   oz < 0 ? B_zm : B_z, oz < 0 ? B_z : B_zp, am_a, vh, Ihp, php);
            }
            if (ok_b) {
                const int mwb = mwa + kMW;
                const int oz = cell_off(__float_as_int(A_z[mwb]), 0);
                transport_complete(g, dt, b, z, yb, x, mwb, A_z, B_zm, B_z, B_zp,
                                   oz < 0 ? B_zm : B_z, oz < 0 ? B_z : B_zp, am_b, vh, Ihp, php);
            }
        }
        am_a = a0_a;
        a0_a = ap_a;
        ap_a = make_float2(0.f, 0.f);
        am_b = a0_b;
        a0_b = ap_b;
        ap_b = make_float2(0.f, 0.f);
    }
    if constexpr (K::kPersistent) {
        kb.sync();  // every wait on the barriers has returned
        if (tid == 0) {
            mbar_inval(&bar[0]);
            mbar_inval(&bar[1]);
        }
    }
}


#ifndef META_BODIES_ONLY
__global__ void __launch_bounds__(kMThreads, 4)
k_adj_transport3d(const __grid_constant__ CUtensorMap tmRecA, const __grid_constant__ CUtensorMap tmRecD, const __grid_constant__ CUtensorMap tmSt, Geom g, Coefs cf, int t, Slots sl, int zc, const float* __restrict__ states, const unsigned int* __restrict__ maxdisp, const float* __restrict__ rec, float* vh, float* Ihp, float* php, unsigned int* fault) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_adj_transport3d<HwBlk>(HwBlk{}, tmRecA, tmRecD, tmSt, g, cf, t, sl, zc, states, maxdisp, rec, vh, Ihp, php, fault);
}
#endif

// Shared tail of the gradp kernels.  mode 0: the record of step t-1; mode 3:
// raw I^_t, p^_t into rawI / rawP (step t-1 lies in a forward segment that is
// recomputed first); at t = 0, mode 1: the cost gradient, mode 2: the
// shooting adjoint.
template <int NDIM, bool PDET>
__device__ __forceinline__ void gradp_tail(const Geom& g, const Coefs& cf, int t, int mode,
                                           const Slots& sl, const Vox& v, long long o, float Ihv,
                                           float phv, float kg, float p0v, const float* states,
                                           const float* u, float* rec, float* rawI, float* rawP,
                                           float* out0, float* gI0) {
    if (mode == 0) {
        build_record<NDIM, PDET>(g, cf, sl.st1, sl.ut1, v, o, Ihv, phv, states, u, rec);
    } else if (mode == 3) {
        rawI[(long long)v.b * g.inst + o] = Ihv;
        rawP[(long long)v.b * g.inst + o] = phv;
    } else {
        const long long ci = cidx(g, v);
        if (mode == 1) {
            const float lam = cf.lambda[v.b], rho = cf.rho[v.b];
            // every rounding explicit: the same bits from every kernel that runs
            // this tail (a contraction into FMAs is free to differ between them)
            const float reg = __fadd_rn(__fmul_rn(2.f, kg), __fmul_rn(__fmul_rn(2.f, rho), p0v));
            out0[ci] = __fadd_rn(phv, __fmul_rn(lam, reg));
        } else {
            out0[ci] = phv;
            if (gI0) gI0[ci] = Ihv;
        }
    }
}

// 2-D adj_gradp on a 32 x 16 tile, two rows per thread (y and y + 8): m^
// (both components), I_t and p_t staged with a one-voxel halo by cp.async.  When the record of step t-1 has R = 1,
// u_{t-1} and p_{t-1} are staged too and the record is built from them (the
// same expressions as build_record).
template <class K, bool PDET>
__device__ __forceinline__ void body_adj_gradp2d(const K& kb, Geom g, Coefs cf, int t, int mode, Slots sl, const float* states, const float* u, const unsigned int* maxdisp, const float* mh, float* Ihp, float* php, float* rec, float* rawI, float* rawP, float* out0, float* gI0) {
    constexpr int TY = 2 * kPY, W = kPX + 8, HR = TY + 2;
    float* sM0 = reinterpret_cast<float*>(kb.smem());
    float* sM1 = sM0 + HR * W;
    float* sI = sM1 + HR * W;
    float* sP = sI + HR * W;
    float* sU0 = sP + HR * W;
    float* sU1 = sU0 + HR * W;
    float* sPp = sU1 + HR * W;
    const int b = kb.bz();
    const int x0 = kb.bx() * kPX, y0 = kb.by() * TY;
    const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
    const float* m0 = mh + (long long)b * g.inst;
    const float* m1 = mh + ((long long)g.B + b) * g.inst;
    const int Rprev = (t > 0) ? gather_radius(maxdisp, t - 1, g.B, b) : 0;
    const bool staged_rec = (mode == 0) && Rprev == 1;  // uniform over the CTA
    stage_async<W, HR>(sM0, m0, g, x0 - 4, y0 - 1, kb.ty() * kPX + kb.tx());
    stage_async<W, HR>(sM1, m1, g, x0 - 4, y0 - 1, kb.ty() * kPX + kb.tx());
    stage_async<W, HR>(sI, It, g, x0 - 4, y0 - 1, kb.ty() * kPX + kb.tx());
    stage_async<W, HR>(sP, pt, g, x0 - 4, y0 - 1, kb.ty() * kPX + kb.tx());
    if (staged_rec) {
        stage_async<W, HR>(sU0, slice_of(u, g, ((long long)sl.ut1 * 2 + 0) * g.B + b), g,
                           x0 - 4, y0 - 1, kb.ty() * kPX + kb.tx());
        stage_async<W, HR>(sU1, slice_of(u, g, ((long long)sl.ut1 * 2 + 1) * g.B + b), g,
                           x0 - 4, y0 - 1, kb.ty() * kPX + kb.tx());
        stage_async<W, HR>(sPp, slice_of(states, g, ((long long)sl.st1 * 2 + 1) * g.B + b), g,
                           x0 - 4, y0 - 1, kb.ty() * kPX + kb.tx());
    }
    cp_async_wait_all();
    kb.sync();
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int ty = kb.ty() + rr * kPY;
        Vox v;
        v.b = b;
        v.x = x0 + kb.tx();
        v.y = y0 + ty;
        v.z = 0;
        v.ok = v.x < g.nx && v.y < g.ny;
        if (!v.ok) continue;
        const int x = v.x, y = v.y;
        const int o = y * g.P + x;
        const long long ob = (long long)b * g.inst + o;
        const int c = (ty + 1) * W + kb.tx() + 4;
        float phv = php[ob];
        float Ihv = Ihp[ob];
        if (Rprev > GatherTile<2>::RMAX) {
            Ihp[ob] = 0.f;  // the next (earlier) step scatters into these
            php[ob] = 0.f;
        }
        // axis 0 (y): stride W in the staged tile
        // roundings explicit: the same bits from every kernel that runs this body
        const float g0 = 0.5f * (sI[c + (y < g.ny - 1 ? W : 0)] - sI[c - (y > 0 ? W : 0)]);
        phv = __fmaf_rn(sM0[c], g0, phv);
        {
            float r = 0.f;
            if (y >= 1) r = __fmaf_rn(0.5f, __fmul_rn(sM0[c - W], sP[c - W]), r);
            if (y == g.ny - 1) r = __fmaf_rn(0.5f, __fmul_rn(sM0[c], sP[c]), r);
            if (y <= g.ny - 2) r = __fmaf_rn(-0.5f, __fmul_rn(sM0[c + W], sP[c + W]), r);
            if (y == 0) r = __fmaf_rn(-0.5f, __fmul_rn(sM0[c], sP[c]), r);
            Ihv = __fadd_rn(Ihv, r);
        }
        // axis 1 (x)
        const float g1 = 0.5f * (sI[c + (x < g.nx - 1 ? 1 : 0)] - sI[c - (x > 0 ? 1 : 0)]);
        phv = __fmaf_rn(sM1[c], g1, phv);
        {
            float r = 0.f;
            if (x >= 1) r = __fmaf_rn(0.5f, __fmul_rn(sM1[c - 1], sP[c - 1]), r);
            if (x == g.nx - 1) r = __fmaf_rn(0.5f, __fmul_rn(sM1[c], sP[c]), r);
            if (x <= g.nx - 2) r = __fmaf_rn(-0.5f, __fmul_rn(sM1[c + 1], sP[c + 1]), r);
            if (x == 0) r = __fmaf_rn(-0.5f, __fmul_rn(sM1[c], sP[c]), r);
            Ihv = __fadd_rn(Ihv, r);
        }
        if (staged_rec) {
            // record of step t-1 from the staged u_{t-1}, p_{t-1}
            const float rho = cf.rho[b], mu = cf.mu[b], dt = cf.dt;
            const float dtrho = dt * rho;
            const float d0 = disp_of(dtrho, sU0[c]), d1 = disp_of(dtrho, sU1[c]);
            const int ys = (y < g.ny - 1 ? W : 0), yl = (y > 0 ? W : 0);
            const int xs = (x < g.nx - 1 ? 1 : 0), xl = (x > 0 ? 1 : 0);
            float fac;  // div v, or (PDET) det(Id - dt Dv)
            if constexpr (PDET) {
                const float A[2][2] = {
                    {rn_cdiff(sU0[c + ys], sU0[c - yl]), rn_cdiff(sU0[c + xs], sU0[c - xl])},
                    {rn_cdiff(sU1[c + ys], sU1[c - yl]), rn_cdiff(sU1[c + xs], sU1[c - xl])}};
                fac = rn_jac_det<2>(A, dtrho);
            } else {
                float du = 0.f;
                du = __fadd_rn(du, rn_cdiff(sU0[c + ys], sU0[c - yl]));
                du = __fadd_rn(du, rn_cdiff(sU1[c + xs], sU1[c - xl]));
                fac = __fmul_rn(-rho, du);
            }
            const Foot1 fy = foot1g(g, y, d0, g.ny), fx = foot1g(g, x, d1, g.nx);
            const int off[3] = {fy.i0 - y, fx.i0 - x, 0};
            const bool ins[3] = {fy.inside, fx.inside, false};
            const float pw = rn_bilin(sPp + c + off[0] * W + off[1], W, fy.f, fx.f);
            const long long rsl = (long long)g.B * g.inst;
            float* r = rec + ob;
            r[Rec<2>::kCell * rsl] = __int_as_float(pack_cell(off, ins));
            r[rsl] = fy.f;
            r[2 * rsl] = fx.f;
            r[Rec<2>::kI * rsl] = Ihv;
            r[Rec<2>::kP * rsl] = PDET ? rn_ptilde_hat_J(phv, Ihv, dt, mu, fac)
                                       : rn_ptilde_hat(phv, Ihv, dt, mu, fac);
            r[Rec<2>::kD * rsl] = rn_div_hat(dt, pw, phv);
            continue;
        }
        float kg = 0.f;
        if (t == 0 && mode == 1) {
            kg = __fmaf_rn(g0, slice_of(u, g, ((long long)sl.u0 * 2 + 0) * g.B + b)[o], kg);
            kg = __fmaf_rn(g1, slice_of(u, g, ((long long)sl.u0 * 2 + 1) * g.B + b)[o], kg);
        }
        gradp_tail<2, PDET>(g, cf, t, mode, sl, v, o, Ihv, phv, kg, sP[c], states, u, rec, rawI,
                            rawP, out0, gI0);
    }
}


#ifndef META_BODIES_ONLY
template <bool PDET>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_gradp2d(Geom g, Coefs cf, int t, int mode, Slots sl, const float* __restrict__ states, const float* __restrict__ u, const unsigned int* __restrict__ maxdisp, const float* __restrict__ mh, float* Ihp, float* php, float* rec, float* rawI, float* rawP, float* out0, float* gI0) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_adj_gradp2d<HwBlk, PDET>(HwBlk{}, g, cf, t, mode, sl, states, u, maxdisp, mh, Ihp, php, rec, rawI, rawP, out0, gI0);
}
#endif

template <class K, int NDIM, bool PDET>
__device__ __forceinline__ void body_adj_gradp(const K& kb, Geom g, Coefs cf, int t, int mode, Slots sl, const float* states, const float* u, const unsigned int* maxdisp, const float* mh, float* Ihp, float* php, float* rec, float* rawI, float* rawP, float* out0, float* gI0) {
    const Vox v = vox_of<NDIM>(g, kb);
    if (!v.ok) return;
    const int b = v.b;
    const long long o = gidx(g, v.z, v.y, v.x);
    const long long ob = (long long)b * g.inst + o;
    int c[NDIM], n[NDIM];
    long long s[NDIM];
    axis_info<NDIM>(g, v, c, n, s);
    const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
    float phv = php[ob];
    float Ihv = Ihp[ob];
    if (t > 0 && gather_radius(maxdisp, t - 1, g.B, b) > GatherTile<NDIM>::RMAX) {
        Ihp[ob] = 0.f;  // the next (earlier) step scatters into these
        php[ob] = 0.f;
    }
    float kg = 0.f;  // sum_a g_a u_a (cost gradient at t = 0)
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const float* ma = mh + ((long long)a * g.B + b) * g.inst;
        const float ga = cdiff(It, o, s[a], c[a], n[a]);
        phv = __fmaf_rn(ma[o], ga, phv);
        // D_a^T (m^_a p) at this node (roundings explicit, as in the 2-D kernel)
        float r = 0.f;
        const long long sa = s[a];
        if (c[a] >= 1) r = __fmaf_rn(0.5f, __fmul_rn(ma[o - sa], pt[o - sa]), r);
        if (c[a] == n[a] - 1) r = __fmaf_rn(0.5f, __fmul_rn(ma[o], pt[o]), r);
        if (c[a] <= n[a] - 2) r = __fmaf_rn(-0.5f, __fmul_rn(ma[o + sa], pt[o + sa]), r);
        if (c[a] == 0) r = __fmaf_rn(-0.5f, __fmul_rn(ma[o], pt[o]), r);
        Ihv = __fadd_rn(Ihv, r);
        if (t == 0 && mode == 1)
            kg = __fmaf_rn(ga, slice_of(u, g, ((long long)sl.u0 * NDIM + a) * g.B + b)[o], kg);
    }
    gradp_tail<NDIM, PDET>(g, cf, t, mode, sl, v, o, Ihv, phv, kg, pt[o], states, u, rec, rawI,
                           rawP, out0, gI0);
}


// 3-D adj_gradp with the momentum update p' = p~ (1 - dt div v), two voxels per
// thread: x and x + 1 (x even), a CTA of 16 x 8 threads covering 32 x 8 voxels.
// Each voxel takes exactly the expressions of body_adj_gradp and build_record
// in the same order; the pair only shares its loads (8-byte loads where the
// two voxels read adjacent addresses, the x neighbours x - 1 and x + 2 once)
// and writes its record fields and raw adjoints as 8-byte pairs.
__device__ __forceinline__ float2 ldg2(const float* p) {
    return *reinterpret_cast<const float2*>(p);
}
__device__ __forceinline__ void st2(float* p, float a, float b, bool both) {
    if (both) *reinterpret_cast<float2*>(p) = make_float2(a, b);
    else p[0] = a;
}

template <class K>
__device__ __forceinline__ void body_adj_gradp3_pair(const K& kb, Geom g, Coefs cf, int t, int mode, Slots sl, const float* states, const float* u, const unsigned int* maxdisp, const float* mh, float* Ihp, float* php, float* rec, float* rawI, float* rawP, float* out0, float* gI0) {
    const int nyt = (g.ny + kPY - 1) / kPY;
    const int z = div_nyt(g, kb.by());
    const int y = (kb.by() - z * nyt) * kPY + kb.ty();
    const int x = kb.bx() * kPX + 2 * kb.tx();
    const int b = kb.bz();
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    const bool two = x + 1 < g.nx;  // the pair's second voxel exists
    const long long o = gidx(g, z, y, x);
    const long long ob = (long long)b * g.inst + o;
    const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
    const float2 ph2 = ldg2(php + ob), Ih2 = ldg2(Ihp + ob);
    float phv[2] = {ph2.x, ph2.y}, Ihv[2] = {Ih2.x, Ih2.y};
    if (t > 0 && gather_radius(maxdisp, t - 1, g.B, b) > GatherTile<3>::RMAX) {
        st2(Ihp + ob, 0.f, 0.f, two);  // the next (earlier) step scatters into these
        st2(php + ob, 0.f, 0.f, two);
    }
    const float2 p2 = ldg2(pt + o);
    const float pc[2] = {p2.x, p2.y};
    float kg[2] = {0.f, 0.f};  // sum_a g_a u_a (cost gradient at t = 0)
    const int cz[2] = {z, z}, cy[2] = {y, y};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float* ma = mh + ((long long)a * g.B + b) * g.inst;
        const float2 m2 = ldg2(ma + o);
        const float mc[2] = {m2.x, m2.y};
        float ga[2], r[2] = {0.f, 0.f};
        if (a < 2) {  // z or y: both voxels read the same rows
            const long long sa = a == 0 ? g.slab : (long long)g.P;
            const int c = a == 0 ? cz[0] : cy[0], n = a == 0 ? g.nz : g.ny;
            const long long hi = (c < n - 1) ? sa : 0, lo = (c > 0) ? sa : 0;
            const float2 Ih = ldg2(It + o + hi), Il = ldg2(It + o - lo);
            ga[0] = 0.5f * (Ih.x - Il.x);
            ga[1] = 0.5f * (Ih.y - Il.y);
            float2 mlo = make_float2(0.f, 0.f), plo = mlo, mhi = mlo, phi = mlo;
            if (c >= 1) {
                mlo = ldg2(ma + o - sa);
                plo = ldg2(pt + o - sa);
            }
            if (c <= n - 2) {
                mhi = ldg2(ma + o + sa);
                phi = ldg2(pt + o + sa);
            }
            const float ml[2] = {mlo.x, mlo.y}, pl[2] = {plo.x, plo.y};
            const float mhv[2] = {mhi.x, mhi.y}, phh[2] = {phi.x, phi.y};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (c >= 1) r[k] = __fmaf_rn(0.5f, __fmul_rn(ml[k], pl[k]), r[k]);
                if (c == n - 1) r[k] = __fmaf_rn(0.5f, __fmul_rn(mc[k], pc[k]), r[k]);
                if (c <= n - 2) r[k] = __fmaf_rn(-0.5f, __fmul_rn(mhv[k], phh[k]), r[k]);
                if (c == 0) r[k] = __fmaf_rn(-0.5f, __fmul_rn(mc[k], pc[k]), r[k]);
            }
        } else {  // x: the pair's own columns and the neighbours x - 1, x + 2
            const float2 I2 = ldg2(It + o);
            const float Iw = x > 0 ? It[o - 1] : 0.f;
            const float Ie = x + 2 < g.nx ? It[o + 2] : 0.f;
            ga[0] = 0.5f * ((x < g.nx - 1 ? I2.y : I2.x) - (x > 0 ? Iw : I2.x));
            ga[1] = 0.5f * ((x + 1 < g.nx - 1 ? Ie : I2.y) - I2.x);
            const float mw = x > 0 ? ma[o - 1] : 0.f, pw = x > 0 ? pt[o - 1] : 0.f;
            const float me = x + 2 < g.nx ? ma[o + 2] : 0.f, pe = x + 2 < g.nx ? pt[o + 2] : 0.f;
            // voxel x (c = x)
            if (x >= 1) r[0] = __fmaf_rn(0.5f, __fmul_rn(mw, pw), r[0]);
            if (x == g.nx - 1) r[0] = __fmaf_rn(0.5f, __fmul_rn(mc[0], pc[0]), r[0]);
            if (x <= g.nx - 2) r[0] = __fmaf_rn(-0.5f, __fmul_rn(mc[1], pc[1]), r[0]);
            if (x == 0) r[0] = __fmaf_rn(-0.5f, __fmul_rn(mc[0], pc[0]), r[0]);
            // voxel x + 1 (c = x + 1 >= 1)
            r[1] = __fmaf_rn(0.5f, __fmul_rn(mc[0], pc[0]), r[1]);
            if (x + 1 == g.nx - 1) r[1] = __fmaf_rn(0.5f, __fmul_rn(mc[1], pc[1]), r[1]);
            if (x + 1 <= g.nx - 2) r[1] = __fmaf_rn(-0.5f, __fmul_rn(me, pe), r[1]);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            phv[k] = __fmaf_rn(mc[k], ga[k], phv[k]);
            Ihv[k] = __fadd_rn(Ihv[k], r[k]);
        }
        if (t == 0 && mode == 1) {
            const float2 u2 = ldg2(slice_of(u, g, ((long long)sl.u0 * 3 + a) * g.B + b) + o);
            kg[0] = __fmaf_rn(ga[0], u2.x, kg[0]);
            kg[1] = __fmaf_rn(ga[1], u2.y, kg[1]);
        }
    }
    if (mode == 0) {  // the record of step t-1 (build_record, two voxels)
        const float rho = cf.rho[b], dtrho = cf.dt * rho;
        float d[2][3], du[2] = {0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float* ua = slice_of(u, g, ((long long)sl.ut1 * 3 + a) * g.B + b);
            const float2 uc = ldg2(ua + o);
            d[0][a] = disp_of(dtrho, uc.x);
            d[1][a] = disp_of(dtrho, uc.y);
            float cd[2];
            if (a < 2) {
                const long long sa = a == 0 ? g.slab : (long long)g.P;
                const int c = a == 0 ? z : y, n = a == 0 ? g.nz : g.ny;
                const long long hi = (c < n - 1) ? sa : 0, lo = (c > 0) ? sa : 0;
                const float2 uh = ldg2(ua + o + hi), ul = ldg2(ua + o - lo);
                cd[0] = rn_cdiff(uh.x, ul.x);
                cd[1] = rn_cdiff(uh.y, ul.y);
            } else {
                const float uw = x > 0 ? ua[o - 1] : 0.f;
                const float ue = x + 2 < g.nx ? ua[o + 2] : 0.f;
                cd[0] = rn_cdiff(x < g.nx - 1 ? uc.y : uc.x, x > 0 ? uw : uc.x);
                cd[1] = rn_cdiff(x + 1 < g.nx - 1 ? ue : uc.y, uc.x);
            }
            du[0] = __fadd_rn(du[0], cd[0]);
            du[1] = __fadd_rn(du[1], cd[1]);
        }
        const float* pprev = slice_of(states, g, ((long long)sl.st1 * 2 + 1) * g.B + b);
        Vox v{b, z, y, x, true};
        const RecVals<3> r0 = record_values<3>(g, cf, v, Ihv[0], phv[0], d[0],
                                               __fmul_rn(-rho, du[0]), pprev);
        RecVals<3> r1 = r0;
        if (two) {
            v.x = x + 1;
            r1 = record_values<3>(g, cf, v, Ihv[1], phv[1], d[1], __fmul_rn(-rho, du[1]), pprev);
        }
        const long long sls = (long long)g.B * g.inst;
        float* w = rec + ob;
#pragma unroll
        for (int k = 0; k < 7; ++k) st2(w + k * sls, r0.v[k], r1.v[k], two);
    } else if (mode == 3) {
        st2(rawI + ob, Ihv[0], Ihv[1], two);
        st2(rawP + ob, phv[0], phv[1], two);
    } else {
        const long long ci = (((long long)b * g.nz + z) * g.ny + y) * g.nx + x;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k == 1 && !two) break;
            if (mode == 1) {
                const float lam = cf.lambda[b], rho = cf.rho[b];
                // every rounding explicit, as in gradp_tail
                const float reg = __fadd_rn(__fmul_rn(2.f, kg[k]),
                                            __fmul_rn(__fmul_rn(2.f, rho), pc[k]));
                out0[ci + k] = __fadd_rn(phv[k], __fmul_rn(lam, reg));
            } else {
                out0[ci + k] = phv[k];
                if (gI0) gI0[ci + k] = Ihv[k];
            }
        }
    }
}

#ifndef META_BODIES_ONLY
__global__ void __launch_bounds__(kPX * kPY / 2)
k_adj_gradp3_pair(Geom g, Coefs cf, int t, int mode, Slots sl, const float* __restrict__ states, const float* __restrict__ u, const unsigned int* __restrict__ maxdisp, const float* __restrict__ mh, float* Ihp, float* php, float* rec, float* rawI, float* rawP, float* out0, float* gI0) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_adj_gradp3_pair<HwBlk>(HwBlk{}, g, cf, t, mode, sl, states, u, maxdisp, mh, Ihp, php, rec, rawI, rawP, out0, gI0);
}
#endif

#ifndef META_BODIES_ONLY
template <int NDIM, bool PDET>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_gradp(Geom g, Coefs cf, int t, int mode, Slots sl, const float* __restrict__ states, const float* __restrict__ u, const unsigned int* __restrict__ maxdisp, const float* __restrict__ mh, float* Ihp, float* php, float* rec, float* rawI, float* rawP, float* out0, float* gI0) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_adj_gradp<HwBlk, NDIM, PDET>(HwBlk{}, g, cf, t, mode, sl, states, u, maxdisp, mh, Ihp, php, rec, rawI, rawP, out0, gI0);
}
#endif

// R = cof(M) - Id for M = Id + B, B = dt rho Du at one voxel (the
// derivative of det M is cof M), column e only, written without the
// cancellation of cof - 1 on the diagonal.
template <int NDIM>
__device__ __forceinline__ void cof_minus_id_col(const float (&B)[NDIM][NDIM], int e,
                                                 float* R) {
    if constexpr (NDIM == 2) {
        // cof(M) = [[M11, -M10], [-M01, M00]]
        R[0] = e == 0 ? B[1][1] : -B[1][0];
        R[1] = e == 0 ? -B[0][1] : B[0][0];
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int a1 = a == 0 ? 1 : 0, a2 = a == 2 ? 1 : 2;  // rows other than a
            const int e1 = e == 0 ? 1 : 0, e2 = e == 2 ? 1 : 2;  // columns other than e
            if (a == e) {
                R[a] = B[a1][a1] + B[a2][a2] + (B[a1][a1] * B[a2][a2] - B[a1][a2] * B[a2][a1]);
            } else {
                const float m11 = (a1 == e1 ? 1.f : 0.f) + B[a1][e1];
                const float m22 = (a2 == e2 ? 1.f : 0.f) + B[a2][e2];
                const float m12 = (a1 == e2 ? 1.f : 0.f) + B[a1][e2];
                const float m21 = (a2 == e1 ? 1.f : 0.f) + B[a2][e1];
                const float minor = m11 * m22 - m12 * m21;
                R[a] = ((a + e) & 1) ? -minor : minor;
            }
        }
    }
}

// Adjoint of the det momentum update beyond its first-order part.  With
// M = Id - dt Dv, dJ/dDv_ae = -dt cof(M)_ae, so v^_a receives
// sum_e D_e^T (div^ cof(M)_ae), div^ = -dt p~ p^' (record field kD).  The
// transport added the identity part of cof, D_a^T div^; this kernel adds
// sum_e D_e^T (div^ R_ae), R = cof(M) - Id, evaluating M at the neighbours
// that D_e^T reads from u_t (slot sl.ut), each thread for its own node.
#ifndef META_BODIES_ONLY
template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_jacT(Geom g, Coefs cf, Slots sl, const float* __restrict__ u, const float* __restrict__ rec,
           float* vh) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const int b = v.b;
    const float dtrho = cf.dt * cf.rho[b];
    const long long o = gidx(g, v.z, v.y, v.x);
    int c[NDIM], n[NDIM];
    long long s[NDIM];
    axis_info<NDIM>(g, v, c, n, s);
    const float* ua[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) ua[a] = slice_of(u, g, ((long long)sl.ut * NDIM + a) * g.B + b);
    const float* dh = slice_of(rec, g, (long long)Rec<NDIM>::kD * g.B + b);
    float acc[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) acc[a] = 0.f;
#pragma unroll
    for (int e = 0; e < NDIM; ++e) {
        // D_e^T f at the node: +f/2 from the node below, -f/2 from the node above,
        // and the edge rows of D (replicated neighbour) at the node itself
#pragma unroll
        for (int k = -1; k <= 1; ++k) {
            float w;
            if (k < 0) w = c[e] >= 1 ? 0.5f : 0.f;
            else if (k > 0) w = c[e] <= n[e] - 2 ? -0.5f : 0.f;
            else w = (c[e] == n[e] - 1 ? 0.5f : 0.f) - (c[e] == 0 ? 0.5f : 0.f);
            if (w == 0.f) continue;
            const long long q = o + k * s[e];
            int cq[NDIM];
#pragma unroll
            for (int f = 0; f < NDIM; ++f) cq[f] = c[f] + (f == e ? k : 0);
            float B[NDIM][NDIM];  // dt rho D_f u_a at q
#pragma unroll
            for (int a = 0; a < NDIM; ++a)
#pragma unroll
                for (int f = 0; f < NDIM; ++f) {
                    const long long hi = (cq[f] < n[f] - 1) ? s[f] : 0, lo = (cq[f] > 0) ? s[f] : 0;
                    B[a][f] = dtrho * (0.5f * (ua[a][q + hi] - ua[a][q - lo]));
                }
            float R[NDIM];
            cof_minus_id_col<NDIM>(B, e, R);
            const float wd = w * dh[q];
#pragma unroll
            for (int a = 0; a < NDIM; ++a) acc[a] += wd * R[a];
        }
    }
#pragma unroll
    for (int a = 0; a < NDIM; ++a) slice_of(vh, g, (long long)a * g.B + b)[o] += acc[a];
}
#endif

// Adjoint of one Eulerian step (I' = I - dt sum_a (D_a I) v_a + dt mu p,
// p' = p - dt sum_a D_a (p v_a), v = -rho u_t) up to v, from the raw adjoints
// I^', p^' (rawI, rawP) of step t+1:
//   Ihp = I^' + sum_a D_a^T (-dt I^' v_a)
//   php = p^' + dt mu I^' + sum_a f^_a v_a,    f^_a = -dt D_a^T p^'
//   v^_a = -dt I^' D_a I + f^_a p
// The blur of v^ and k_adj_gradp (raw mode) complete the step.
#ifndef META_BODIES_ONLY
template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_euler_adj(Geom g, Coefs cf, Slots sl, const float* __restrict__ states,
            const float* __restrict__ u, const float* __restrict__ rawI,
            const float* __restrict__ rawP, float* Ihp, float* php, float* vh) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const int b = v.b;
    const float rho = cf.rho[b], mu = cf.mu[b], dt = cf.dt;
    const long long o = gidx(g, v.z, v.y, v.x);
    int c[NDIM], n[NDIM];
    long long s[NDIM];
    axis_info<NDIM>(g, v, c, n, s);
    const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
    const float* RI = slice_of(rawI, g, b);
    const float* RP = slice_of(rawP, g, b);
    const float Ih = RI[o];
    float Inew = Ih, pnew = RP[o] + (dt * mu) * Ih;
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const float* ua = slice_of(u, g, ((long long)sl.ut * NDIM + a) * g.B + b);
        const long long sa = s[a];
        // D_a^T of f = -dt I^' v_a = dt rho I^' u_a at this node
        auto f = [&](long long q) { return (dt * rho) * (RI[q] * ua[q]); };
        float r = 0.f;
        if (c[a] >= 1) r += 0.5f * f(o - sa);
        if (c[a] == n[a] - 1) r += 0.5f * f(o);
        if (c[a] <= n[a] - 2) r -= 0.5f * f(o + sa);
        if (c[a] == 0) r -= 0.5f * f(o);
        Inew += r;
        const float fh = -dt * cdiff_T(RP, o, sa, c[a], n[a]);
        const float va = -rho * ua[o];
        pnew += fh * va;
        const float ga = cdiff(It, o, sa, c[a], n[a]);
        vh[((long long)a * g.B + b) * g.inst + o] = -dt * Ih * ga + fh * pt[o];
    }
    slice_of(Ihp, g, b)[o] = Inew;
    slice_of(php, g, b)[o] = pnew;
}
#endif

// The Eulerian momentum step of the hybrid scheme, transposed, added to what
// the semi-Lagrangian transport left for its image step:
//   php += p^' + sum_a f^_a v_a,   v^_a += f^_a p,   f^_a = -dt D_a^T p^'
#ifndef META_BODIES_ONLY
template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_hybrid_p(Geom g, Coefs cf, Slots sl, const float* __restrict__ states,
           const float* __restrict__ u, const float* __restrict__ rawP, float* php, float* vh) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const int b = v.b;
    const float rho = cf.rho[b], dt = cf.dt;
    const long long o = gidx(g, v.z, v.y, v.x);
    int c[NDIM], n[NDIM];
    long long s[NDIM];
    axis_info<NDIM>(g, v, c, n, s);
    const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
    const float* RP = slice_of(rawP, g, b);
    float pnew = RP[o];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const float* ua = slice_of(u, g, ((long long)sl.ut * NDIM + a) * g.B + b);
        const float fh = -dt * cdiff_T(RP, o, s[a], c[a], n[a]);
        pnew += fh * (-rho * ua[o]);
        vh[((long long)a * g.B + b) * g.inst + o] += fh * pt[o];
    }
    slice_of(php, g, b)[o] += pnew;
}
#endif

}  // namespace

#ifndef META_BODIES_ONLY
// ---------------------------------------------------------------- launchers

cudaError_t launch_cost(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                        const float* states, const float* u, const float* J,
                        const unsigned int* maxdisp, float* rec, float* Ihp, float* php,
                        float* rawI, float* rawP, double* partials, int nblk, double* cost,
                        cudaStream_t st) {
    if (std::vector<PRec>* r = recorder()) {
        PRec e{};
        e.kind = PK_COSTP;
        e.ndim = ndim;
        e.grid = dim3(nblk, g.B);
        e.bx = 256;
        e.by = 1;
        e.smem = kCostSmem;
        e.a.g = g;
        e.a.sl = sl;
        e.a.c[0] = states;
        e.a.c[1] = u;
        e.a.c[2] = J;
        e.a.d[0] = partials;
        r->push_back(e);
        PRec f{};
        f.kind = PK_ADJINIT;
        f.ndim = ndim;
        f.sub = 1;
        f.grid = ndim == 2 ? pgrid<2>(g) : pgrid<3>(g);
        f.bx = kPX;
        f.by = kPY;
        f.a.g = g;
        f.a.cf = c;
        f.a.sl = sl;
        f.a.c[0] = states;
        f.a.c[1] = u;
        f.a.c[2] = J;
        f.a.cmd = maxdisp;
        f.a.w[0] = rec;
        f.a.w[1] = Ihp;
        f.a.w[2] = php;
        f.a.w[3] = rawI;
        f.a.w[4] = rawP;
        r->push_back(f);
        PRec h{};
        h.kind = PK_COSTF;
        h.ndim = ndim;
        h.grid = dim3(g.B);
        h.bx = 256;
        h.by = 1;
        h.smem = kCostSmem;
        h.a.n = nblk;
        h.a.cf = c;
        h.a.d[0] = partials;
        h.a.d[1] = cost;
        r->push_back(h);
        return cudaSuccess;
    }
    const dim3 grid(nblk, g.B);
    const dim3 blk(kPX, kPY);
    if (ndim == 2) {
        META_CHECK_LAUNCH(launch_k(k_cost_partials<2>, grid, 256, kCostSmem, st, g, sl, states, u, J,
                                   partials));
        META_CHECK_LAUNCH(launch_k(k_adj_init<2, true>, pgrid<2>(g), blk, 0, st, g, c, sl, states,
                                   u, J, (const float*)nullptr, maxdisp, rec, Ihp, php, rawI,
                                   rawP));
    } else {
        META_CHECK_LAUNCH(launch_k(k_cost_partials<3>, grid, 256, kCostSmem, st, g, sl, states, u, J,
                                   partials));
        META_CHECK_LAUNCH(launch_k(k_adj_init<3, true>, pgrid<3>(g), blk, 0, st, g, c, sl, states,
                                   u, J, (const float*)nullptr, maxdisp, rec, Ihp, php, rawI,
                                   rawP));
    }
    META_CHECK_LAUNCH(launch_k(k_cost_final, g.B, 256, kCostSmem, st, nblk, c, partials, cost));
    return cudaSuccess;
}

cudaError_t launch_adj_init(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                            const float* states, const float* u, const float* gI1,
                            const float* gp1, const unsigned int* maxdisp, float* rec, float* Ihp,
                            float* php, float* rawI, float* rawP, cudaStream_t st) {
    if (recorder()) return cudaErrorNotSupported;  // not replayable by the persistent kernel
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_adj_init<2, false>, pgrid<2>(g), blk, 0, st, g, c, sl, states,
                                   u, gI1, gp1, maxdisp, rec, Ihp, php, rawI, rawP));
    else
        META_CHECK_LAUNCH(launch_k(k_adj_init<3, false>, pgrid<3>(g), blk, 0, st, g, c, sl, states,
                                   u, gI1, gp1, maxdisp, rec, Ihp, php, rawI, rawP));
    return cudaSuccess;
}

cudaError_t launch_adj_records(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                               const float* states, const float* u, const float* rawI,
                               const float* rawP, float* rec, cudaStream_t st) {
    if (std::vector<PRec>* r = recorder()) {
        PRec e{};
        e.kind = PK_ADJREC;
        e.ndim = ndim;
        e.grid = ndim == 2 ? pgrid<2>(g) : pgrid<3>(g);
        e.bx = kPX;
        e.by = kPY;
        e.a.g = g;
        e.a.cf = c;
        e.a.sl = sl;
        e.a.c[0] = states;
        e.a.c[1] = u;
        e.a.c[2] = rawI;
        e.a.c[3] = rawP;
        e.a.w[0] = rec;
        r->push_back(e);
        return cudaSuccess;
    }
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_adj_records<2>, pgrid<2>(g), blk, 0, st, g, c, sl, states, u,
                                   rawI, rawP, rec));
    else
        META_CHECK_LAUNCH(launch_k(k_adj_records<3>, pgrid<3>(g), blk, 0, st, g, c, sl, states, u,
                                   rawI, rawP, rec));
    return cudaSuccess;
}

cudaError_t launch_adj_transport(const Geom& g, int ndim, const Coefs& c, int t, const Slots& sl,
                                 const CUtensorMap* maps, const float* states,
                                 const unsigned int* maxdisp, const float* rec, float* vh,
                                 float* Ihp, float* php, unsigned int* fault, cudaStream_t st) {
    if (std::vector<PRec>* r = recorder()) {
        PRec e{};
        e.kind = PK_TRANS;
        e.ndim = ndim;
        e.bx = kPX;
        e.by = ndim == 2 ? kPY : kMTY;
        if (ndim == 2) {
            e.grid = gather_grid2d(g);
            e.smem = kTr2dSmem;
        } else {
            const int zc = g.zct > 0 ? g.zct : march_chunk(g, 4, 2, kTransRows);
            e.grid = dim3(((g.nx + 31) / 32) * ((g.nz + zc - 1) / zc),
                          (g.ny + kTransRows - 1) / kTransRows, g.B);
            e.smem = kMarchSmem;
            e.a.zc = zc;
            e.ntm = 3;
            for (int k = 0; k < 3; ++k) e.tm[k] = maps[k];
        }
        e.a.g = g;
        e.a.cf = c;
        e.a.t = t;
        e.a.sl = sl;
        e.a.c[0] = states;
        e.a.cmd = maxdisp;
        e.a.c[1] = rec;
        e.a.w[0] = vh;
        e.a.w[1] = Ihp;
        e.a.w[2] = php;
        e.a.fault = fault;
        r->push_back(e);
        return cudaSuccess;
    }
    if (ndim == 2) {
        META_CHECK_LAUNCH(launch_k(k_adj_transport2d, gather_grid2d(g), dim3(kPX, kPY), kTr2dSmem, st,
                                   g, c, t, sl, states, maxdisp, rec, vh, Ihp, php, fault));
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_adj_transport3d,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kMarchSmem);
        if (e != cudaSuccess) return e;
        const int zc = g.zct > 0 ? g.zct : march_chunk(g, 4, 2, kTransRows);
        const dim3 grid(((g.nx + 31) / 32) * ((g.nz + zc - 1) / zc),
                        (g.ny + kTransRows - 1) / kTransRows, g.B);
        META_CHECK_LAUNCH(launch_k(k_adj_transport3d, grid, dim3(kPX, kMTY), kMarchSmem, st, maps[0], maps[1],
                                   maps[2], g, c, t, sl, zc, states, maxdisp, rec, vh, Ihp, php,
                                   fault));
    }
    return cudaSuccess;
}

cudaError_t launch_adj_gradp(const Geom& g, int ndim, const Coefs& c, int t, int mode,
                             const Slots& sl, const float* states, const float* u,
                             const unsigned int* maxdisp, const float* mh, float* Ihp, float* php,
                             float* rec, float* rawI, float* rawP, float* out0, float* gI0,
                             cudaStream_t st) {
    if (std::vector<PRec>* r = recorder()) {
        PRec e{};
        e.kind = PK_GRADP;
        e.ndim = ndim;
        e.sub = c.pdet;
        e.bx = kPX;
        e.by = kPY;
        if (ndim == 2) {
            e.grid = dim3((g.nx + kPX - 1) / kPX, (g.ny + 2 * kPY - 1) / (2 * kPY), g.B);
            e.smem = kGradp2dSmem;
        } else {
            e.grid = pgrid<3>(g);
            if (!c.pdet) e.bx = kPX / 2;  // two voxels per thread
        }
        e.a.g = g;
        e.a.cf = c;
        e.a.t = t;
        e.a.mode = mode;
        e.a.sl = sl;
        e.a.c[0] = states;
        e.a.c[1] = u;
        e.a.cmd = maxdisp;
        e.a.c[2] = mh;
        e.a.w[0] = Ihp;
        e.a.w[1] = php;
        e.a.w[2] = rec;
        e.a.w[3] = rawI;
        e.a.w[4] = rawP;
        e.a.w[5] = out0;
        e.a.w[6] = gI0;
        r->push_back(e);
        return cudaSuccess;
    }
    const dim3 blk(kPX, kPY);
    if (ndim == 2) {
        const dim3 grid((g.nx + kPX - 1) / kPX, (g.ny + 2 * kPY - 1) / (2 * kPY), g.B);
        META_CHECK_LAUNCH(launch_k(c.pdet ? k_adj_gradp2d<true> : k_adj_gradp2d<false>, grid, blk,
                                   kGradp2dSmem, st, g, c, t, mode, sl, states, u, maxdisp, mh, Ihp, php,
                                   rec, rawI, rawP, out0, gI0));
    } else if (c.pdet) {
        META_CHECK_LAUNCH(launch_k(k_adj_gradp<3, true>, pgrid<3>(g), blk, 0, st, g, c, t, mode,
                                   sl, states, u, maxdisp, mh, Ihp, php, rec, rawI, rawP, out0,
                                   gI0));
    } else {
        META_CHECK_LAUNCH(launch_k(k_adj_gradp3_pair, pgrid<3>(g), dim3(kPX / 2, kPY), 0, st, g, c,
                                   t, mode, sl, states, u, maxdisp, mh, Ihp, php, rec, rawI, rawP,
                                   out0, gI0));
    }
    return cudaSuccess;
}

cudaError_t launch_adj_jacT(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                            const float* u, const float* rec, float* vh, cudaStream_t st) {
    if (recorder()) return cudaErrorNotSupported;  // not replayable by the persistent kernel
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_adj_jacT<2>, pgrid<2>(g), blk, 0, st, g, c, sl, u, rec, vh));
    else
        META_CHECK_LAUNCH(launch_k(k_adj_jacT<3>, pgrid<3>(g), blk, 0, st, g, c, sl, u, rec, vh));
    return cudaSuccess;
}

cudaError_t launch_euler_adj(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                             const float* states, const float* u, const float* rawI,
                             const float* rawP, float* Ihp, float* php, float* vh,
                             cudaStream_t st) {
    if (recorder()) return cudaErrorNotSupported;  // not replayable by the persistent kernel
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_euler_adj<2>, pgrid<2>(g), blk, 0, st, g, c, sl, states, u,
                                   rawI, rawP, Ihp, php, vh));
    else
        META_CHECK_LAUNCH(launch_k(k_euler_adj<3>, pgrid<3>(g), blk, 0, st, g, c, sl, states, u,
                                   rawI, rawP, Ihp, php, vh));
    return cudaSuccess;
}

cudaError_t launch_hybrid_p(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                            const float* states, const float* u, const float* rawP, float* php,
                            float* vh, cudaStream_t st) {
    if (recorder()) return cudaErrorNotSupported;  // not replayable by the persistent kernel
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_hybrid_p<2>, pgrid<2>(g), blk, 0, st, g, c, sl, states, u,
                                   rawP, php, vh));
    else
        META_CHECK_LAUNCH(launch_k(k_hybrid_p<3>, pgrid<3>(g), blk, 0, st, g, c, sl, states, u,
                                   rawP, php, vh));
    return cudaSuccess;
}

#endif  // META_BODIES_ONLY

}  // namespace meta
