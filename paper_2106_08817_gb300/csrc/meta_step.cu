// meta_step.cu -- the forward semi-Lagrangian step (arXiv:2106.08817, Eq. 3
// integrated as in Sec. 2.3), sm_103a.  After the blur passes have produced
// u_t = K(p_t grad I_t) (v_t = -rho u_t):
//   k_advect2d / k_advect3d  div v, foot y = x - dt v, bi/trilinear gathers of
//       I_t and p_t, p_{t+1} = p~ (1 - dt div v), I_{t+1} = I~ + dt mu p~, and
//       the per-instance max displacement (the window of the adjoint), or with
//       the det update p_{t+1} = p~ det(Id - dt Dv); 2-D on
//       staged 32 x 8 tiles, 3-D marching along z through a ring of planes.
//   k_euler  the Eulerian and hybrid steps of Sec. 2.3 (their adjoints are in
//       meta_adjoint.cu).
//   k_deform / k_deform_out  the deformation phi_t of the grid and det D phi_T.
//   k_pack / k_unpack  copies between the caller's contiguous arrays and the
//       pitched trajectory.
#include "meta_stencil.cuh"

namespace meta {

namespace {

// ------------------------------------------------------------------ kernels

template <class K, int NDIM>
__device__ __forceinline__ void body_pack(const K& kb, Geom g, const float* I0, const float* p0, float* dI, float* dP) {
    const Vox v = vox_of<NDIM>(g, kb);
    if (!v.ok) return;
    const long long o = (long long)v.b * g.inst + gidx(g, v.z, v.y, v.x);
    const long long ci = cidx(g, v);
    dI[o] = I0[ci];
    dP[o] = p0[ci];
}


#ifndef META_BODIES_ONLY
template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_pack(Geom g, const float* __restrict__ I0, const float* __restrict__ p0, float* dI, float* dP) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_pack<HwBlk, NDIM>(HwBlk{}, g, I0, p0, dI, dP);
}
#endif

#ifndef META_BODIES_ONLY
template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_unpack(Geom g, const float* __restrict__ sI, const float* __restrict__ sP, float* I1, float* p1) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const long long o = (long long)v.b * g.inst + gidx(g, v.z, v.y, v.x);
    const long long ci = cidx(g, v);
    if (I1) I1[ci] = sI[o];
    if (p1) p1[ci] = sP[o];
}
#endif

// 2-D advect on a 32 x 16 tile, two rows per thread (y and y + 8): u staged
// with a one-voxel halo, I_t and p_t with a four-voxel halo (feet whose cell
// leaves it read global memory).
constexpr int kAdvHalo = 4;
constexpr int kAdvTY = 2 * kPY;  // rows per tile
constexpr int kAdvW = kPX + 2 * kAdvHalo;      // 40: staged row length
constexpr int kAdvHU = kAdvTY + 2;             // 18: staged rows of u
constexpr int kAdvHI = kAdvTY + 2 * kAdvHalo;  // 24: staged rows of I, p
// dynamic shared memory of the 2-D advect: u (two components), I_t, p_t
constexpr int kAdv2dSmem = (2 * kAdvHU + 2 * kAdvHI) * kAdvW * 4;

template <class K, bool PDET>
__device__ __forceinline__ void body_advect2d(const K& kb, Geom g, Coefs cf, int t, Slots sl, float* __restrict__ states, const float* __restrict__ u, unsigned int* __restrict__ maxdisp) {
    constexpr int W = kAdvW, HU = kAdvHU, HI = kAdvHI;
    float* sU0 = reinterpret_cast<float*>(kb.smem());
    float* sU1 = sU0 + HU * W;
    float* sI = sU1 + HU * W;
    float* sP = sI + HI * W;
    const int b = kb.bz();
    const int x0 = kb.bx() * kPX, y0 = kb.by() * kAdvTY;
    const float* u0 = slice_of(u, g, ((long long)sl.ut * 2 + 0) * g.B + b);
    const float* u1 = slice_of(u, g, ((long long)sl.ut * 2 + 1) * g.B + b);
    const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
    stage_async<W, HU>(sU0, u0, g, x0 - kAdvHalo, y0 - 1, kb.ty() * kPX + kb.tx());
    stage_async<W, HU>(sU1, u1, g, x0 - kAdvHalo, y0 - 1, kb.ty() * kPX + kb.tx());
    stage_async<W, HI>(sI, It, g, x0 - kAdvHalo, y0 - kAdvHalo, kb.ty() * kPX + kb.tx());
    stage_async<W, HI>(sP, pt, g, x0 - kAdvHalo, y0 - kAdvHalo, kb.ty() * kPX + kb.tx());
    cp_async_wait_all();
    kb.sync();
    const int x = x0 + kb.tx();
    float dmax = 0.f;
    const float rho = cf.rho[b], mu = cf.mu[b], dt = cf.dt;
    const float dtrho = dt * rho;
    float* I1 = slice_of(states, g, ((long long)sl.st1 * 2 + 0) * g.B + b);
    float* p1 = slice_of(states, g, ((long long)sl.st1 * 2 + 1) * g.B + b);
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int ty = kb.ty() + rr * kPY;
        const int y = y0 + ty;
        if (x >= g.nx || y >= g.ny) continue;
        const int ui = (ty + 1) * W + kb.tx() + kAdvHalo;
        const float d0 = disp_of(dtrho, sU0[ui]);
        const float d1 = disp_of(dtrho, sU1[ui]);
        float du = 0.f;
        du += 0.5f * (sU0[ui + (y < g.ny - 1 ? W : 0)] - sU0[ui - (y > 0 ? W : 0)]);
        du += 0.5f * (sU1[ui + (x < g.nx - 1 ? 1 : 0)] - sU1[ui - (x > 0 ? 1 : 0)]);
        dmax = fmaxf(dmax, fmaxf(fabsf(d0), fabsf(d1)));
        const float div = -rho * du;
        float jac = 0.f;  // PDET: det(Id - dt Dv)
        if constexpr (PDET) {
            const int ys = y < g.ny - 1 ? W : 0, yl = y > 0 ? W : 0;
            const int xs = x < g.nx - 1 ? 1 : 0, xl = x > 0 ? 1 : 0;
            const float A[2][2] = {
                {rn_cdiff(sU0[ui + ys], sU0[ui - yl]), rn_cdiff(sU0[ui + xs], sU0[ui - xl])},
                {rn_cdiff(sU1[ui + ys], sU1[ui - yl]), rn_cdiff(sU1[ui + xs], sU1[ui - xl])}};
            jac = rn_jac_det<2>(A, dtrho);
        }
        const Foot1 fy = foot1g(g, y, d0, g.ny), fx = foot1g(g, x, d1, g.nx);
        const int ly = fy.i0 - (y0 - kAdvHalo), lx = fx.i0 - (x0 - kAdvHalo);
        float Iw, pw;
        if (ly >= 0 && ly + 1 < HI && lx >= 0 && lx + 1 < W) {
            Iw = bilin(sI + ly * W + lx, W, fy.f, fx.f);
            pw = bilin(sP + ly * W + lx, W, fy.f, fx.f);
        } else {
            const int o = fy.i0 * g.P + fx.i0;
            Iw = bilin(It + o, g.P, fy.f, fx.f);
            pw = bilin(pt + o, g.P, fy.f, fx.f);
        }
        const int o = y * g.P + x;
        p1[o] = PDET ? pw * jac : pw * (1.f - dt * div);
        I1[o] = Iw + (dt * mu) * pw;
    }
    // one atomic per CTA (per-warp atomics on one word per instance serialise in L2)
    __shared__ unsigned int s_m;
    if (kb.tx() == 0 && kb.ty() == 0) s_m = 0u;
    kb.sync();
    const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
    if ((kb.tx() & 31) == 0 && m != 0u) atomicMax(&s_m, m);
    kb.sync();
    if (kb.tx() == 0 && kb.ty() == 0 && s_m != 0u)
        atomicMax(maxdisp + kMaxdispStride * ((long long)t * g.B + b), s_m);
}


#ifndef META_BODIES_ONLY
template <bool PDET>
__global__ void __launch_bounds__(kPX * kPY)
k_advect2d(Geom g, Coefs cf, int t, Slots sl, float* __restrict__ states, const float* __restrict__ u, unsigned int* __restrict__ maxdisp) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_advect2d<HwBlk, PDET>(HwBlk{}, g, cf, t, sl, states, u, maxdisp);
}
#endif

// 3-D advect: a CTA owns a 32 x kAR (12) column over planes [zs, zs + zc) and
// marches along z; each thread computes two adjacent rows (x, y0 + 2 ty) and
// (x, y0 + 2 ty + 1).  Plane p of u (three components) and of I_t, p_t, with
// a one-voxel y halo and x in [x0 - 4, x0 + 36), arrives by TMA (two tiled
// copies from 5-D tensor maps over the u and state stacks, issued by one
// thread, completing on an mbarrier per plane parity) into a ring of 4 plane
// slots: plane p + 1 is in flight while the voxels of plane p - 1 are computed
// from planes p - 2 .. p.  Planes outside the volume are never read, so none
// is copied for them.  Feet whose cell leaves the staged window (per-step
// displacements of a voxel or more) read global memory.
constexpr int kAR = kAdvRows;                         // rows of a CTA's column (two per thread)
constexpr int kAW = 40, kAH = kAR + 2, kAPL = kAW * kAH;  // staged window (x, y) of a plane
constexpr int kAUF = (3 * kAPL * 4 + 127) / 128 * 128 / 4;  // u fields of a slot, 128-byte multiple
constexpr int kASlot = kAUF + 2 * kAPL;              // then I_t, p_t
constexpr int kARing = 4;                            // plane slots
constexpr size_t kAdvMarchSmem = 128 + (size_t)kARing * kASlot * sizeof(float);
constexpr uint32_t kABytes = 5 * kAPL * 4;           // bytes of one staged plane
static_assert((kAUF * 4) % 128 == 0 && (kASlot * 4) % 128 == 0 && kAUF >= 3 * kAPL,
              "TMA destinations start on 128-byte boundaries");

// The 3-D advect's arithmetic, every rounding explicit (no contraction), in the
// expressions the adjoint's record builder uses: div v_t as -rho times the sum
// of the central differences of u (rn_cdiff, summed over z, y, x), the
// interpolated I and p by rn_lerp along x, then y, then z, p' = p~ (1 - dt div)
// and I' = I~ + (dt mu) p~.  The forward therefore computes exactly the div and p~
// that the records of the same step recompute.  Two rows (a pair) run the same
// per-lane operations on packed FP32 pairs; one row runs them scalar.

// Window index offsets of the central differences of row y (a row of the staged
// window is kAW floats).
__device__ __forceinline__ void adv_du_offsets(const Geom& g, int y, int x, int* yh, int* yl,
                                               int* xh, int* xl) {
    *yh = y < g.ny - 1 ? kAW : 0;
    *yl = y > 0 ? kAW : 0;
    *xh = x < g.nx - 1 ? 1 : 0;
    *xl = x > 0 ? 1 : 0;
}

// Interpolated (I, p) at a foot from the staged window (planes pl, ph) or global memory.
__device__ __forceinline__ float2 adv_interp(const Geom& g, const Foot1& fz, const Foot1& fy,
                                             const Foot1& fx, int z, int y0, int x0,
                                             const float* sm1, const float* s0,
                                             const float* sp1, const float* It,
                                             const float* pt) {
    const int kz = fz.i0 - (z - 1), ky = fy.i0 - (y0 - 1), kx = fx.i0 - (x0 - 4);
    if (kz >= 0 && kz + 1 < 3 && ky >= 0 && ky + 1 < kAH && kx >= 0 && kx + 1 < kAW) {
        const float* pl = kz == 0 ? sm1 : s0;
        const float* ph = kz == 0 ? s0 : sp1;
        const float* lo = pl + kAUF + ky * kAW + kx;
        const float* hi = ph + kAUF + ky * kAW + kx;
        return make_float2(rn_trilin(lo, hi, kAW, fz.f, fy.f, fx.f),
                           rn_trilin(lo + kAPL, hi + kAPL, kAW, fz.f, fy.f, fx.f));
    }
    const long long gi = gidx(g, fz.i0, fy.i0, fx.i0);
    return make_float2(rn_trilin(It + gi, It + gi + g.slab, g.P, fz.f, fy.f, fx.f),
                       rn_trilin(pt + gi, pt + gi + g.slab, g.P, fz.f, fy.f, fx.f));
}

// One voxel (row y, window index ui) from the staged planes sm1, s0, sp1 (z - 1,
// z, z + 1).
template <bool PDET>
__device__ __forceinline__ void advect3d_voxel(const Geom& g, float rho, float mu, float dt,
                                               float dtrho, int z, int y, int x, int y0, int x0,
                                               int ui, const float* sm1, const float* s0,
                                               const float* sp1, const float* It,
                                               const float* pt, float* I1, float* p1,
                                               float& dmax) {
    const float* u0 = s0;
    const float* u1 = s0 + kAPL;
    const float* u2 = s0 + 2 * kAPL;
    int yh, yl, xh, xl;
    adv_du_offsets(g, y, x, &yh, &yl, &xh, &xl);
    const float d0 = __fmul_rn(dtrho, u0[ui]), d1 = __fmul_rn(dtrho, u1[ui]),
                d2 = __fmul_rn(dtrho, u2[ui]);
    float du = 0.f;
    du = __fadd_rn(du, rn_cdiff(z < g.nz - 1 ? sp1[ui] : u0[ui], z > 0 ? sm1[ui] : u0[ui]));
    du = __fadd_rn(du, rn_cdiff(u1[ui + yh], u1[ui - yl]));
    du = __fadd_rn(du, rn_cdiff(u2[ui + xh], u2[ui - xl]));
    dmax = fmaxf(dmax, fmaxf(fabsf(d0), fmaxf(fabsf(d1), fabsf(d2))));
    float fac;  // 1 - dt div v, or det(Id - dt Dv) for the det update
    if constexpr (PDET) {
        float A[3][3];  // A[a][e] = D_e u_a
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float* c0 = s0 + a * kAPL;
            A[a][0] = rn_cdiff(z < g.nz - 1 ? sp1[a * kAPL + ui] : c0[ui],
                               z > 0 ? sm1[a * kAPL + ui] : c0[ui]);
            A[a][1] = rn_cdiff(c0[ui + yh], c0[ui - yl]);
            A[a][2] = rn_cdiff(c0[ui + xh], c0[ui - xl]);
        }
        fac = rn_jac_det<3>(A, dtrho);
    } else {
        fac = __fsub_rn(1.f, __fmul_rn(dt, __fmul_rn(-rho, du)));
    }
    const Foot1 fz = foot1g(g, z, d0, g.nz), fy = foot1g(g, y, d1, g.ny), fx = foot1g(g, x, d2, g.nx);
    const float2 w = adv_interp(g, fz, fy, fx, z, y0, x0, sm1, s0, sp1, It, pt);
    const long long o = gidx(g, z, y, x);
    p1[o] = __fmul_rn(w.y, fac);
    I1[o] = __fadd_rn(w.x, __fmul_rn(__fmul_rn(dt, mu), w.y));
}

// Packed rn_lerp: (1 - f) a + f b per lane.
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 f, float2 omf) {
    return fadd2(fmul2(omf, a), fmul2(f, b));
}
// Packed rn_trilin of two voxels whose corners start at pa / qa and pb / qb
// (lower and upper plane, row stride kAW).
__device__ __forceinline__ float2 trilin2(const float* pa, const float* qa, const float* pb,
                                          const float* qb, float2 fz, float2 fy, float2 fx,
                                          float2 oz, float2 oy, float2 ox) {
    const float2 b0 = lerp2(lerp2(make_float2(pa[0], pb[0]), make_float2(pa[1], pb[1]), fx, ox),
                            lerp2(make_float2(pa[kAW], pb[kAW]),
                                  make_float2(pa[kAW + 1], pb[kAW + 1]), fx, ox),
                            fy, oy);
    const float2 b1 = lerp2(lerp2(make_float2(qa[0], qb[0]), make_float2(qa[1], qb[1]), fx, ox),
                            lerp2(make_float2(qa[kAW], qb[kAW]),
                                  make_float2(qa[kAW + 1], qb[kAW + 1]), fx, ox),
                            fy, oy);
    return lerp2(b0, b1, fz, oz);
}

// Rows y and y + 1 (window indices ui and ui + kAW) of the same column: the
// operations of advect3d_voxel (momentum update p~ (1 - dt div v)) on packed
// pairs, lane 0 the first row, lane 1 the second.
__device__ __forceinline__ void advect3d_pair(const Geom& g, float rho, float mu, float dt,
                                              float dtrho, int z, int y, int x, int y0, int x0,
                                              int ui, const float* sm1, const float* s0,
                                              const float* sp1, const float* It,
                                              const float* pt, float* I1, float* p1,
                                              float& dmax) {
    const float* u0 = s0;
    const float* u1 = s0 + kAPL;
    const float* u2 = s0 + 2 * kAPL;
    const int ub = ui + kAW;
    int yha, yla, xh, xl, yhb, ylb;
    adv_du_offsets(g, y, x, &yha, &yla, &xh, &xl);
    adv_du_offsets(g, y + 1, x, &yhb, &ylb, &xh, &xl);
    const float2 dr = make_float2(dtrho, dtrho);
    const float2 d0 = fmul2(dr, make_float2(u0[ui], u0[ub]));
    const float2 d1 = fmul2(dr, make_float2(u1[ui], u1[ub]));
    const float2 d2 = fmul2(dr, make_float2(u2[ui], u2[ub]));
    const float2 half = make_float2(0.5f, 0.5f);
    const float* zh = z < g.nz - 1 ? sp1 : u0;
    const float* zl = z > 0 ? sm1 : u0;
    float2 du = make_float2(0.f, 0.f);
    du = fadd2(du, fmul2(half, fsub2(make_float2(zh[ui], zh[ub]), make_float2(zl[ui], zl[ub]))));
    du = fadd2(du, fmul2(half, fsub2(make_float2(u1[ui + yha], u1[ub + yhb]),
                                     make_float2(u1[ui - yla], u1[ub - ylb]))));
    du = fadd2(du, fmul2(half, fsub2(make_float2(u2[ui + xh], u2[ub + xh]),
                                     make_float2(u2[ui - xl], u2[ub - xl]))));
    dmax = fmaxf(dmax, fmaxf(fmaxf(fabsf(d0.x), fabsf(d0.y)),
                             fmaxf(fmaxf(fabsf(d1.x), fabsf(d1.y)),
                                   fmaxf(fabsf(d2.x), fabsf(d2.y)))));
    const float2 one = make_float2(1.f, 1.f);
    const float2 fac = fsub2(one, fmul2(make_float2(dt, dt),
                                        fmul2(make_float2(-rho, -rho), du)));
    const Foot1 fza = foot1g(g, z, d0.x, g.nz), fya = foot1g(g, y, d1.x, g.ny), fxa = foot1g(g, x, d2.x, g.nx);
    const Foot1 fzb = foot1g(g, z, d0.y, g.nz), fyb = foot1g(g, y + 1, d1.y, g.ny),
                fxb = foot1g(g, x, d2.y, g.nx);
    const int kza = fza.i0 - (z - 1), kya = fya.i0 - (y0 - 1), kxa = fxa.i0 - (x0 - 4);
    const int kzb = fzb.i0 - (z - 1), kyb = fyb.i0 - (y0 - 1), kxb = fxb.i0 - (x0 - 4);
    const bool sa = kza >= 0 && kza + 1 < 3 && kya >= 0 && kya + 1 < kAH && kxa >= 0 &&
                    kxa + 1 < kAW;
    const bool sb = kzb >= 0 && kzb + 1 < 3 && kyb >= 0 && kyb + 1 < kAH && kxb >= 0 &&
                    kxb + 1 < kAW;
    float2 Iw, pw;
    if (sa && sb) {  // both feet inside the staged window: one packed interpolation
        const float2 fz = make_float2(fza.f, fzb.f), fy = make_float2(fya.f, fyb.f),
                     fx = make_float2(fxa.f, fxb.f);
        const float2 oz = fsub2(one, fz), oy = fsub2(one, fy), ox = fsub2(one, fx);
        const float* pa = (kza == 0 ? sm1 : s0) + kAUF + kya * kAW + kxa;
        const float* qa = (kza == 0 ? s0 : sp1) + kAUF + kya * kAW + kxa;
        const float* pb = (kzb == 0 ? sm1 : s0) + kAUF + kyb * kAW + kxb;
        const float* qb = (kzb == 0 ? s0 : sp1) + kAUF + kyb * kAW + kxb;
        Iw = trilin2(pa, qa, pb, qb, fz, fy, fx, oz, oy, ox);
        pw = trilin2(pa + kAPL, qa + kAPL, pb + kAPL, qb + kAPL, fz, fy, fx, oz, oy, ox);
    } else {
        const float2 wa = adv_interp(g, fza, fya, fxa, z, y0, x0, sm1, s0, sp1, It, pt);
        const float2 wb = adv_interp(g, fzb, fyb, fxb, z, y0, x0, sm1, s0, sp1, It, pt);
        Iw = make_float2(wa.x, wb.x);
        pw = make_float2(wa.y, wb.y);
    }
    const float2 pn = fmul2(pw, fac);
    const float dm = __fmul_rn(dt, mu);
    const float2 In = fadd2(Iw, fmul2(make_float2(dm, dm), pw));
    const long long o = gidx(g, z, y, x);
    p1[o] = pn.x;
    I1[o] = In.x;
    p1[o + g.P] = pn.y;
    I1[o + g.P] = In.y;
}

template <class K, bool PDET>
__device__ __forceinline__ void body_advect3d(const K& kb, const CUtensorMap& tmU, const CUtensorMap& tmS, Geom g, Coefs cf, int t, Slots sl, int zc, float* __restrict__ states, unsigned int* __restrict__ maxdisp, unsigned int* fault) {
    unsigned char* smem_raw = kb.smem();
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // [2]: planes of even / odd index
    float* ring = reinterpret_cast<float*>(smem_raw + 128);
    const int b = kb.bz();
    const int nxc = (g.nx + 31) / 32;
    const int x0 = (kb.bx() % nxc) * 32;
    const int zs = (kb.bx() / nxc) * zc;
    const int ze = min(zs + zc, g.nz);
    const int y0 = kb.by() * kAR;
    const int tx = kb.tx(), ty = kb.ty();
    const int tid = ty * kPX + tx;
    const int x = x0 + tx, ya = y0 + 2 * ty, yb = ya + 1;
    const bool ok_a = x < g.nx && ya < g.ny, ok_b = x < g.nx && yb < g.ny;
    const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
    float* I1 = slice_of(states, g, ((long long)sl.st1 * 2 + 0) * g.B + b);
    float* p1 = slice_of(states, g, ((long long)sl.st1 * 2 + 1) * g.B + b);
    // plane p sits in slot (p - zs + 1) mod 4
    auto slot = [&](int p) { return ring + ((p - zs + 1) & 3) * kASlot; };
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        if constexpr (K::kPersistent) {
            tmap_acquire(&tmU);
            tmap_acquire(&tmS);
            fence_proxy_async_global();
        }
    }
    kb.sync();
    auto load_plane = [&](int p) {
        uint64_t* br = &bar[(p - zs + 1) & 1];
        if (p >= 0 && p < g.nz) {
            mbar_arrive_expect_tx(br, kABytes);
            float* dst = slot(p);
            tma_load_5d(dst, &tmU, br, x0 - 4, y0 - 1, p, b, 3 * sl.ut);
            tma_load_5d(dst + kAUF, &tmS, br, x0 - 4, y0 - 1, p, b, 2 * sl.st);
        } else {
            mbar_arrive(br);
        }
    };
    const float rho = cf.rho[b], mu = cf.mu[b], dt = cf.dt;
    const float dtrho = dt * rho;
    const int uia = (2 * ty + 1) * kAW + tx + 4;  // window index of row a in a plane
    float dmax = 0.f;
    // every warp waits (bounded) for each plane itself, so one CTA barrier per plane
    // suffices; a wait that runs out raises s_fail, which all threads read after the
    // next barrier and leave together
    __shared__ int s_fail;
    if (tid == 0) {
        s_fail = 0;
        load_plane(zs - 1);
    }
    int p = zs - 1;
    for (; p <= ze; ++p) {
        const int j = p - zs + 1;  // planes staged so far
        kb.sync();  // every read of the slot plane p + 1 reuses is done; s_fail is seen
        if (s_fail) break;
        if (tid == 0 && p + 1 <= ze) load_plane(p + 1);
        if (!mbar_wait_bounded(&bar[j & 1], (j >> 1) & 1, fault)) {
            s_fail = 1;
            continue;
        }
        const int z = p - 1;  // planes z - 1 .. z + 1 are staged
        if (z < zs) continue;
        const float* sm1 = slot(z - 1);
        const float* s0 = slot(z);
        const float* sp1 = slot(z + 1);
        if (!PDET && ok_a && ok_b) {
            advect3d_pair(g, rho, mu, dt, dtrho, z, ya, x, y0, x0, uia, sm1, s0, sp1, It, pt, I1,
                          p1, dmax);
        } else {
            if (ok_a)
                advect3d_voxel<PDET>(g, rho, mu, dt, dtrho, z, ya, x, y0, x0, uia, sm1, s0, sp1,
                                     It, pt, I1, p1, dmax);
            if (ok_b)
                advect3d_voxel<PDET>(g, rho, mu, dt, dtrho, z, yb, x, y0, x0, uia + kAW, sm1, s0,
                                     sp1, It, pt, I1, p1, dmax);
        }
    }
    if (p <= ze && tid < 32) {  // left after a wait ran out at plane p - 1: the copy of
        const int j = p - zs + 1;  // plane p may still be in flight, so let it land
        mbar_wait_bounded(&bar[j & 1], (j >> 1) & 1, fault, 100000000ull);  // (bounded)
    }
    // one atomic per CTA (per-warp atomics on one word per instance serialise in L2)
    __shared__ unsigned int s_m;
    if (tid == 0) s_m = 0u;
    kb.sync();
    if (!s_fail) {
        const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
        if ((tid & 31) == 0 && m != 0u) atomicMax(&s_m, m);
    }
    kb.sync();
    if (tid == 0 && s_m != 0u) atomicMax(maxdisp + kMaxdispStride * ((long long)t * g.B + b), s_m);
    if constexpr (K::kPersistent) {
        if (tid == 0) {  // every wait on the barriers has returned (the barrier above)
            mbar_inval(&bar[0]);
            mbar_inval(&bar[1]);
        }
    }
}


#ifndef META_BODIES_ONLY
template <bool PDET>
__global__ void __launch_bounds__(kPX * kPY)
k_advect3d(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmS, Geom g, Coefs cf, int t, Slots sl, int zc, float* __restrict__ states, unsigned int* __restrict__ maxdisp, unsigned int* fault) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    body_advect3d<HwBlk, PDET>(HwBlk{}, tmU, tmS, g, cf, t, sl, zc, states, maxdisp, fault);
}
#endif

// Eulerian (HYBRID = false) and hybrid steps of Sec. 2.3.  With
// v = -rho u (slot sl.ut) and the central differences D of the scheme:
//   p' = p - dt sum_a D_a (p v_a)                       (conservative Eq. 7)
//   I' = I - dt sum_a (D_a I) v_a + dt mu p             (Eq. 5, Eulerian)
//   I' = I~ + dt mu p~ at the foot of the advect         (hybrid)
// from state slot sl.st into sl.st1.  Plain L1-cached loads of the 2d
// neighbours.  The hybrid records its per-step max displacement, the gather
// window of its adjoint's image step; the Eulerian adjoint needs none.
#ifndef META_BODIES_ONLY
template <int NDIM, bool HYBRID>
__global__ void __launch_bounds__(kPX * kPY)
k_euler(Geom g, Coefs cf, int t, Slots sl, float* __restrict__ states,
        const float* __restrict__ u, unsigned int* __restrict__ maxdisp) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    const Vox v = vox_of<NDIM>(g);
    float dmax = 0.f;  // hybrid: max |d| of the CTA (the window of its adjoint transport)
    if (v.ok) {
        const int b = v.b;
        const float rho = cf.rho[b], mu = cf.mu[b], dt = cf.dt;
        const long long o = gidx(g, v.z, v.y, v.x);
        int c[NDIM], n[NDIM];
        long long s[NDIM];
        axis_info<NDIM>(g, v, c, n, s);
        const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
        const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
        float* I1 = slice_of(states, g, ((long long)sl.st1 * 2 + 0) * g.B + b);
        float* p1 = slice_of(states, g, ((long long)sl.st1 * 2 + 1) * g.B + b);
        float divpv = 0.f, adv = 0.f, d[NDIM];
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const float* ua = slice_of(u, g, ((long long)sl.ut * NDIM + a) * g.B + b);
            const long long hi = (c[a] < n[a] - 1) ? s[a] : 0, lo = (c[a] > 0) ? s[a] : 0;
            divpv += 0.5f * (pt[o + hi] * (-rho * ua[o + hi]) - pt[o - lo] * (-rho * ua[o - lo]));
            if constexpr (HYBRID) d[a] = disp_of(dt * rho, ua[o]);
            else adv += (0.5f * (It[o + hi] - It[o - lo])) * (-rho * ua[o]);
        }
        p1[o] = pt[o] - dt * divpv;
        if constexpr (HYBRID) {
            const Feet<NDIM> F = feet_of<NDIM>(g, v, d);
            const float pw = interp<NDIM>(g, F, pt);
            I1[o] = interp<NDIM>(g, F, It) + (dt * mu) * pw;
#pragma unroll
            for (int a = 0; a < NDIM; ++a) dmax = fmaxf(dmax, fabsf(d[a]));
        } else {
            I1[o] = It[o] - dt * adv + (dt * mu) * pt[o];
        }
    }
    if constexpr (HYBRID) {  // one atomic per CTA, as in the advect
        __shared__ unsigned int s_m;
        const int tid = threadIdx.y * kPX + threadIdx.x;
        if (tid == 0) s_m = 0u;
        __syncthreads();
        const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
        if ((tid & 31) == 0 && m != 0u) atomicMax(&s_m, m);
        __syncthreads();
        if (tid == 0 && s_m != 0u)
            atomicMax(maxdisp + kMaxdispStride * ((long long)t * g.B + blockIdx.z), s_m);
    }
}
#endif

// Deformation of the grid (the deformation grids of Fig. 1-2, Sec. 3): phi_0 = Id and
// phi_{t+1} = phi_t o (Id - dt v_t), i.e. phi_{t+1}(x) = S(y) phi_t at the same
// clamped foot y as the advect of step t.  Kept as the displacement
// w_t = phi_t - Id: the multilinear interpolant reproduces Id at a clamped foot,
// so w_{t+1}(x) = (y - x) + S(y) w_t.  w_t is slice a * B + b of win (NULL at
// t = 0, where w_0 = 0), w_{t+1} goes to the same slices of wout.
#ifndef META_BODIES_ONLY
template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_deform(Geom g, Coefs cf, int su, const float* __restrict__ u, const float* __restrict__ win,
         float* __restrict__ wout) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const int b = v.b;
    const float dtrho = cf.dt * cf.rho[b];
    const long long o = gidx(g, v.z, v.y, v.x);
    float d[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a)
        d[a] = disp_of(dtrho, slice_of(u, g, ((long long)su * NDIM + a) * g.B + b)[o]);
    const Feet<NDIM> F = feet_of<NDIM>(g, v, d);
    int c[NDIM], n[NDIM];
    long long s[NDIM];
    axis_info<NDIM>(g, v, c, n, s);
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        float w = (float)(F.f[a].i0 - c[a]) + F.f[a].f;  // y - x on axis a
        if (win) w += interp<NDIM>(g, F, slice_of(win, g, (long long)a * g.B + b));
        slice_of(wout, g, (long long)a * g.B + b)[o] = w;
    }
}
#endif

// The deformation out of the pitched w = phi - Id: phi (contiguous
// [B][NDIM][N], nullable) = w, and jac (contiguous [B][N], nullable) =
// det(D phi) = det(Id + D w), D the central difference inside and the
// one-sided difference at the two edges of each axis.
#ifndef META_BODIES_ONLY
template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_deform_out(Geom g, const float* __restrict__ w, float* __restrict__ phi,
             float* __restrict__ jac) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const int b = v.b;
    const long long o = gidx(g, v.z, v.y, v.x);
    const long long N = (long long)g.nz * g.ny * g.nx;
    const long long xi = cidx(g, v) - (long long)b * N;  // voxel index in the instance
    int c[NDIM], n[NDIM];
    long long s[NDIM];
    axis_info<NDIM>(g, v, c, n, s);
    float A[NDIM][NDIM];  // A[a][e] = d phi_a / d x_e
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const float* wa = slice_of(w, g, (long long)a * g.B + b);
        if (phi) phi[((long long)b * NDIM + a) * N + xi] = wa[o];
#pragma unroll
        for (int e = 0; e < NDIM; ++e) {
            const long long hi = (c[e] < n[e] - 1) ? s[e] : 0, lo = (c[e] > 0) ? s[e] : 0;
            const float h = (hi != 0 && lo != 0) ? 0.5f : 1.f;
            A[a][e] = (a == e ? 1.f : 0.f) + h * (wa[o + hi] - wa[o - lo]);
        }
    }
    if (!jac) return;
    float det;
    if constexpr (NDIM == 2) {
        det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    } else {
        det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
              A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
              A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    }
    jac[(long long)b * N + xi] = det;
}
#endif

}  // namespace

#ifndef META_BODIES_ONLY
// ---------------------------------------------------------------- launchers

cudaError_t launch_pack(const Geom& g, int ndim, const float* I0, const float* p0, float* dI,
                        float* dP, cudaStream_t st) {
    if (std::vector<PRec>* r = recorder()) {
        PRec e{};
        e.kind = PK_PACK;
        e.ndim = ndim;
        e.grid = ndim == 2 ? pgrid<2>(g) : pgrid<3>(g);
        e.bx = kPX;
        e.by = kPY;
        e.a.g = g;
        e.a.c[0] = I0;
        e.a.c[1] = p0;
        e.a.w[0] = dI;
        e.a.w[1] = dP;
        r->push_back(e);
        return cudaSuccess;
    }
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_pack<2>, pgrid<2>(g), blk, 0, st, g, I0, p0, dI, dP));
    else
        META_CHECK_LAUNCH(launch_k(k_pack<3>, pgrid<3>(g), blk, 0, st, g, I0, p0, dI, dP));
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Geom& g, int ndim, const float* sI, const float* sP, float* I1,
                          float* p1, cudaStream_t st) {
    if (recorder()) return cudaErrorNotSupported;  // not replayable by the persistent kernel
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_unpack<2>, pgrid<2>(g), blk, 0, st, g, sI, sP, I1, p1));
    else
        META_CHECK_LAUNCH(launch_k(k_unpack<3>, pgrid<3>(g), blk, 0, st, g, sI, sP, I1, p1));
    return cudaGetLastError();
}

cudaError_t launch_advect(const Geom& g, int ndim, const Coefs& c, int t, const Slots& sl,
                          float* states, const float* u, unsigned int* maxdisp,
                          const CUtensorMap* maps, unsigned int* fault, cudaStream_t st) {
    // 3-D: plane chunks of the 32 x kAR columns (5 CTAs per SM, 2 staged halo planes)
    const int zc = ndim == 3 ? (g.zca > 0 ? g.zca : march_chunk(g, 5, 2, kAR)) : 1;
    const dim3 grid3(((g.nx + 31) / 32) * ((g.nz + zc - 1) / zc), (g.ny + kAR - 1) / kAR, g.B);
    if (std::vector<PRec>* r = recorder()) {
        PRec e{};
        e.kind = PK_ADVECT;
        e.ndim = ndim;
        e.sub = c.pdet;
        e.bx = kPX;
        e.by = kPY;
        if (ndim == 2) {
            e.grid = dim3((g.nx + kPX - 1) / kPX, (g.ny + kAdvTY - 1) / kAdvTY, g.B);
            e.smem = kAdv2dSmem;
        } else {
            e.grid = grid3;
            e.by = kAR / 2;
            e.smem = kAdvMarchSmem;
            e.a.zc = zc;
            e.ntm = 2;
            e.tm[0] = maps[0];
            e.tm[1] = maps[1];
            e.a.fault = fault;
        }
        e.a.g = g;
        e.a.cf = c;
        e.a.t = t;
        e.a.sl = sl;
        e.a.w[0] = states;
        e.a.c[0] = u;
        e.a.md = maxdisp;
        r->push_back(e);
        return cudaSuccess;
    }
    const dim3 blk(kPX, kPY);
    if (ndim == 2) {
        const dim3 grid((g.nx + kPX - 1) / kPX, (g.ny + kAdvTY - 1) / kAdvTY, g.B);
        META_CHECK_LAUNCH(launch_k(c.pdet ? k_advect2d<true> : k_advect2d<false>, grid, blk,
                                   kAdv2dSmem, st,
                                   g, c, t, sl, states, u, maxdisp));
    } else {
        auto kern = c.pdet ? k_advect3d<true> : k_advect3d<false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kAdvMarchSmem);
        if (e != cudaSuccess) return e;
        META_CHECK_LAUNCH(launch_k(kern, grid3, dim3(kPX, kAR / 2), kAdvMarchSmem, st, maps[0],
                                   maps[1], g, c, t, sl, zc, states, maxdisp, fault));
    }
    return cudaGetLastError();
}

cudaError_t launch_deform(const Geom& g, int ndim, const Coefs& c, int su, const float* u,
                          const float* win, float* wout, cudaStream_t st) {
    if (recorder()) return cudaErrorNotSupported;  // not replayable by the persistent kernel
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_deform<2>, pgrid<2>(g), blk, 0, st, g, c, su, u, win, wout));
    else
        META_CHECK_LAUNCH(launch_k(k_deform<3>, pgrid<3>(g), blk, 0, st, g, c, su, u, win, wout));
    return cudaGetLastError();
}

cudaError_t launch_deform_out(const Geom& g, int ndim, const float* w, float* phi, float* jac,
                              cudaStream_t st) {
    if (recorder()) return cudaErrorNotSupported;  // not replayable by the persistent kernel
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_deform_out<2>, pgrid<2>(g), blk, 0, st, g, w, phi, jac));
    else
        META_CHECK_LAUNCH(launch_k(k_deform_out<3>, pgrid<3>(g), blk, 0, st, g, w, phi, jac));
    return cudaGetLastError();
}

cudaError_t launch_euler(const Geom& g, int ndim, const Coefs& c, int t, const Slots& sl,
                         bool hybrid, float* states, const float* u, unsigned int* maxdisp,
                         cudaStream_t st) {
    if (recorder()) return cudaErrorNotSupported;  // not replayable by the persistent kernel
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(hybrid ? k_euler<2, true> : k_euler<2, false>, pgrid<2>(g), blk,
                                   0, st, g, c, t, sl, states, u, maxdisp));
    else
        META_CHECK_LAUNCH(launch_k(hybrid ? k_euler<3, true> : k_euler<3, false>, pgrid<3>(g), blk,
                                   0, st, g, c, t, sl, states, u, maxdisp));
    return cudaGetLastError();
}

#endif  // META_BODIES_ONLY

}  // namespace meta
