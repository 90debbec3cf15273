// meta_step.cu -- the forward semi-Lagrangian step (arXiv:2106.08817, Eq. 3
// integrated as in Sec. 2.3), sm_103a.  After the blur passes have produced
// u_t = K(p_t grad I_t) (v_t = -rho u_t):
//   k_advect / k_advect2d  div v, foot y = x - dt v, bi/trilinear gathers of
//       I_t and p_t, p_{t+1} = p~ (1 - dt div v), I_{t+1} = I~ + dt mu p~, and
//       the per-instance max displacement (the window of the adjoint).
//   k_pack / k_unpack  copies between the caller's contiguous arrays and the
//       pitched trajectory.
#include "meta_stencil.cuh"

namespace meta {

namespace {

// ------------------------------------------------------------------ kernels

template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_pack(Geom g, const float* __restrict__ I0, const float* __restrict__ p0, float* dI, float* dP) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const long long o = (long long)v.b * g.inst + gidx(g, v.z, v.y, v.x);
    const long long ci = cidx(g, v);
    dI[o] = I0[ci];
    dP[o] = p0[ci];
}

template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_unpack(Geom g, const float* __restrict__ sI, const float* __restrict__ sP, float* I1, float* p1) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const long long o = (long long)v.b * g.inst + gidx(g, v.z, v.y, v.x);
    const long long ci = cidx(g, v);
    if (I1) I1[ci] = sI[o];
    if (p1) p1[ci] = sP[o];
}

// 2-D advect on a 32 x 8 tile: u staged with a one-voxel halo, I_t and p_t
// with a four-voxel halo (feet whose cell leaves it read global memory).
constexpr int kAdvHalo = 4;

__global__ void __launch_bounds__(kPX * kPY)
k_advect2d(Geom g, Coefs cf, int t, Slots sl, float* __restrict__ states,
           const float* __restrict__ u, unsigned int* __restrict__ maxdisp) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    constexpr int W = kPX + 2 * kAdvHalo;        // 40
    constexpr int HU = kPY + 2;                  // 10
    constexpr int HI = kPY + 2 * kAdvHalo;       // 16
    __shared__ __align__(16) float sU0[HU * W], sU1[HU * W], sI[HI * W], sP[HI * W];
    const int b = blockIdx.z;
    const int x0 = blockIdx.x * kPX, y0 = blockIdx.y * kPY;
    const float* u0 = slice_of(u, g, ((long long)sl.ut * 2 + 0) * g.B + b);
    const float* u1 = slice_of(u, g, ((long long)sl.ut * 2 + 1) * g.B + b);
    const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
    stage_async<W, HU>(sU0, u0, g, x0 - kAdvHalo, y0 - 1);
    stage_async<W, HU>(sU1, u1, g, x0 - kAdvHalo, y0 - 1);
    stage_async<W, HI>(sI, It, g, x0 - kAdvHalo, y0 - kAdvHalo);
    stage_async<W, HI>(sP, pt, g, x0 - kAdvHalo, y0 - kAdvHalo);
    cp_async_wait_all();
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    float dmax = 0.f;
    if (x < g.nx && y < g.ny) {
        const float rho = cf.rho[b], mu = cf.mu[b], dt = cf.dt;
        const float dtrho = dt * rho;
        const int ui = (threadIdx.y + 1) * W + threadIdx.x + kAdvHalo;
        const float d0 = disp_of(dtrho, sU0[ui]);
        const float d1 = disp_of(dtrho, sU1[ui]);
        float du = 0.f;
        du += 0.5f * (sU0[ui + (y < g.ny - 1 ? W : 0)] - sU0[ui - (y > 0 ? W : 0)]);
        du += 0.5f * (sU1[ui + (x < g.nx - 1 ? 1 : 0)] - sU1[ui - (x > 0 ? 1 : 0)]);
        dmax = fmaxf(fabsf(d0), fabsf(d1));
        const float div = -rho * du;
        const Foot1 fy = foot1(y, d0, g.ny), fx = foot1(x, d1, g.nx);
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
        float* I1 = slice_of(states, g, ((long long)sl.st1 * 2 + 0) * g.B + b);
        float* p1 = slice_of(states, g, ((long long)sl.st1 * 2 + 1) * g.B + b);
        p1[o] = pw * (1.f - dt * div);
        I1[o] = Iw + (dt * mu) * pw;
    }
    // one atomic per CTA (per-warp atomics on one word per instance serialise in L2)
    __shared__ unsigned int s_m;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_m = 0u;
    __syncthreads();
    const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
    if ((threadIdx.x & 31) == 0 && m != 0u) atomicMax(&s_m, m);
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && s_m != 0u)
        atomicMax(maxdisp + kMaxdispStride * ((long long)t * g.B + b), s_m);
}

template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_advect(Geom g, Coefs cf, int t, Slots sl, float* __restrict__ states,
         const float* __restrict__ u, unsigned int* __restrict__ maxdisp) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    const Vox v = vox_of<NDIM>(g);
    float dmax = 0.f;
    if (v.ok) {
        const int b = v.b;
        const float rho = cf.rho[b], mu = cf.mu[b], dt = cf.dt;
        const float dtrho = dt * rho;
        const long long o = gidx(g, v.z, v.y, v.x);
        int c[NDIM], n[NDIM];
        long long s[NDIM];
        axis_info<NDIM>(g, v, c, n, s);
        float d[NDIM];
        float du = 0.f;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const float* ua = slice_of(u, g, ((long long)sl.ut * NDIM + a) * g.B + b);
            d[a] = disp_of(dtrho, ua[o]);
            du += cdiff(ua, o, s[a], c[a], n[a]);
            dmax = fmaxf(dmax, fabsf(d[a]));
        }
        const float div = -rho * du;  // div v, v = -rho u
        const Feet<NDIM> F = feet_of<NDIM>(g, v, d);
        const float* It = slice_of(states, g, ((long long)sl.st * 2 + 0) * g.B + b);
        const float* pt = slice_of(states, g, ((long long)sl.st * 2 + 1) * g.B + b);
        const float Iw = interp<NDIM>(g, F, It);
        const float pw = interp<NDIM>(g, F, pt);
        float* I1 = slice_of(states, g, ((long long)sl.st1 * 2 + 0) * g.B + b);
        float* p1 = slice_of(states, g, ((long long)sl.st1 * 2 + 1) * g.B + b);
        p1[o] = pw * (1.f - dt * div);
        I1[o] = Iw + (dt * mu) * pw;
    }
    // per-instance max |displacement| (non-negative floats order like their bits),
    // one atomic per CTA
    __shared__ unsigned int s_m;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_m = 0u;
    __syncthreads();
    const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
    if ((threadIdx.x & 31) == 0 && m != 0u) atomicMax(&s_m, m);
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0 && s_m != 0u)
        atomicMax(maxdisp + kMaxdispStride * ((long long)t * g.B + blockIdx.z), s_m);
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_pack(const Geom& g, int ndim, const float* I0, const float* p0, float* dI,
                        float* dP, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_pack<2>, pgrid<2>(g), blk, 0, st, g, I0, p0, dI, dP));
    else
        META_CHECK_LAUNCH(launch_k(k_pack<3>, pgrid<3>(g), blk, 0, st, g, I0, p0, dI, dP));
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Geom& g, int ndim, const float* sI, const float* sP, float* I1,
                          float* p1, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_unpack<2>, pgrid<2>(g), blk, 0, st, g, sI, sP, I1, p1));
    else
        META_CHECK_LAUNCH(launch_k(k_unpack<3>, pgrid<3>(g), blk, 0, st, g, sI, sP, I1, p1));
    return cudaGetLastError();
}

cudaError_t launch_advect(const Geom& g, int ndim, const Coefs& c, int t, const Slots& sl,
                          float* states, const float* u, unsigned int* maxdisp, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_advect2d, dim3((g.nx + kPX - 1) / kPX, (g.ny + kPY - 1) / kPY, g.B), blk, 0, st, g, c, t, sl, states, u, maxdisp));
    else
        META_CHECK_LAUNCH(launch_k(k_advect<3>, pgrid<3>(g), blk, 0, st, g, c, t, sl, states, u, maxdisp));
    return cudaGetLastError();
}

}  // namespace meta
