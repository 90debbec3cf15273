// meta_step.cu -- pointwise and gather kernels of the semi-Lagrangian step and
// of its discrete adjoint (arXiv:2106.08817, Eq. 3-4, Sec. 2.3), sm_103a.
//
// Forward step t (after the blur passes have produced u_t = K(p_t grad I_t)):
//   k_advect      div v, foot y = x - dt v (v = -rho u), bi/trilinear gathers of
//                 I_t and p_t, p_{t+1} = p~ (1 - dt div v), I_{t+1} = I~ + dt mu p~,
//                 and the per-instance max displacement (window of the adjoint).
// Adjoint step t (reverse), the transpose of the step above:
//   k_adj_transport  per source x of a tile and its halo:
//                 p~^ = p^'(1 - dt div v) + dt mu I^', div^ = -dt p~ p^' and the
//                 foot record (shared memory); per node n: S^T by gather over the
//                 sources whose foot cell touches n (fixed order, no atomics), the
//                 foot derivative y^, and v^ = -dt y^ + D^T div^
//   (blur of v^ with K = K^T, scaled by -rho, in meta_blur.cu)
//   k_adj_gradp   p^ += sum_i m^_i D_i I,  I^ += sum_i D_i^T (m^_i p)
// Cost (Eq. 4): k_cost_partials + k_cost_final, FP64 partials in a fixed tree.
#include "meta_kernels.h"

namespace meta {

namespace {

constexpr int kPX = 32, kPY = 8;  // pointwise block

struct Vox {
    int b, z, y, x;
    bool ok;
};

template <int NDIM>
__device__ __forceinline__ Vox vox_of(const Geom& g) {
    Vox v;
    const int nyt = (g.ny + kPY - 1) / kPY;
    v.b = blockIdx.z;
    v.x = blockIdx.x * kPX + threadIdx.x;
    v.y = (blockIdx.y % nyt) * kPY + threadIdx.y;
    v.z = (NDIM == 3) ? (int)(blockIdx.y / nyt) : 0;
    v.ok = v.x < g.nx && v.y < g.ny && v.z < g.nz;
    return v;
}

template <int NDIM>
dim3 pgrid(const Geom& g) {
    return dim3((g.nx + kPX - 1) / kPX, ((g.ny + kPY - 1) / kPY) * g.nz, g.B);
}

__device__ __forceinline__ long long cidx(const Geom& g, const Vox& v) {
    return (((long long)v.b * g.nz + v.z) * g.ny + v.y) * g.nx + v.x;
}

__device__ __forceinline__ const float* slice_of(const float* base, const Geom& g, long long s) {
    return base + s * g.inst;
}
__device__ __forceinline__ float* slice_of(float* base, const Geom& g, long long s) {
    return base + s * g.inst;
}

// Displacement of the foot along one axis, y - x = -dt v = (dt rho) u.  The
// forward step and every adjoint kernel call exactly this expression, so the
// gather-form transpose sees bit-identical feet.
__device__ __forceinline__ float disp_of(float dtrho, float u) { return dtrho * u; }

// Central difference of f at linear offset o along a stride s, edge replicated.
__device__ __forceinline__ float cdiff(const float* f, long long o, long long s, int c, int n) {
    const long long hi = (c < n - 1) ? s : 0;
    const long long lo = (c > 0) ? s : 0;
    return 0.5f * (f[o + hi] - f[o - lo]);
}

// Stages rows [ylo, ylo + ROWS) x columns [xlo, xlo + W) of one pitched slice
// into shared memory (row stride W) with asynchronous 16-byte copies; parts
// outside the slice are zero-filled.  xlo and W are multiples of 4, so every
// 16-byte chunk lies inside one padded row.  All copies of a CTA are in flight
// together; call cp_async_wait_all() and __syncthreads() before reading.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(valid ? 16u : 0u)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <int W, int ROWS>
__device__ __forceinline__ void stage_async(float* dst, const float* __restrict__ src,
                                            const Geom& g, int xlo, int ylo) {
    constexpr int NC4 = W / 4;
    const int tid = threadIdx.y * kPX + threadIdx.x;
    for (int i = tid; i < ROWS * NC4; i += kPX * kPY) {
        const int r = i / NC4, c = i - r * NC4;
        const int y = ylo + r, x = xlo + 4 * c;
        const bool ok = (y >= 0 && y < g.ny && x >= 0 && x < g.P);
        cp_async16(dst + r * W + 4 * c, ok ? src + y * g.P + x : src, ok);
    }
}

// Bilinear value (and derivatives) at lower corner p[0] with row stride W;
// the same expressions as interp / interp_grad below.
__device__ __forceinline__ float bilin(const float* p, int W, float fy, float fx) {
    const float a = (1.f - fx) * p[0] + fx * p[1];
    const float b = (1.f - fx) * p[W] + fx * p[W + 1];
    return (1.f - fy) * a + fy * b;
}
__device__ __forceinline__ void bilin_grad(const float* p, int W, float fy, float fx, bool iny,
                                           bool inx, float* dy, float* dx) {
    const float c00 = p[0], c01 = p[1], c10 = p[W], c11 = p[W + 1];
    const float a = (1.f - fx) * c00 + fx * c01;
    const float b = (1.f - fx) * c10 + fx * c11;
    *dy = iny ? (b - a) : 0.f;
    *dx = inx ? ((1.f - fy) * (c01 - c00) + fy * (c11 - c10)) : 0.f;
}

template <int NDIM>
struct Feet {
    Foot1 f[NDIM];
    long long base;  // linear offset of the lower corner
};

template <int NDIM>
__device__ __forceinline__ Feet<NDIM> feet_of(const Geom& g, const Vox& v, const float* d) {
    Feet<NDIM> F;
    if constexpr (NDIM == 2) {
        F.f[0] = foot1(v.y, d[0], g.ny);
        F.f[1] = foot1(v.x, d[1], g.nx);
        F.base = gidx(g, 0, F.f[0].i0, F.f[1].i0);
    } else {
        F.f[0] = foot1(v.z, d[0], g.nz);
        F.f[1] = foot1(v.y, d[1], g.ny);
        F.f[2] = foot1(v.x, d[2], g.nx);
        F.base = gidx(g, F.f[0].i0, F.f[1].i0, F.f[2].i0);
    }
    return F;
}

// Multilinear interpolant of `f` at the feet.
template <int NDIM>
__device__ __forceinline__ float interp(const Geom& g, const Feet<NDIM>& F, const float* f) {
    const float* p = f + F.base;
    if constexpr (NDIM == 2) {
        const float fy = F.f[0].f, fx = F.f[1].f;
        const float a = (1.f - fx) * p[0] + fx * p[1];
        const float b = (1.f - fx) * p[g.P] + fx * p[g.P + 1];
        return (1.f - fy) * a + fy * b;
    } else {
        const float fz = F.f[0].f, fy = F.f[1].f, fx = F.f[2].f;
        const long long S = g.slab, P = g.P;
        const float a0 = (1.f - fx) * p[0] + fx * p[1];
        const float a1 = (1.f - fx) * p[P] + fx * p[P + 1];
        const float a2 = (1.f - fx) * p[S] + fx * p[S + 1];
        const float a3 = (1.f - fx) * p[S + P] + fx * p[S + P + 1];
        const float b0 = (1.f - fy) * a0 + fy * a1;
        const float b1 = (1.f - fy) * a2 + fy * a3;
        return (1.f - fz) * b0 + fz * b1;
    }
}

// Value and the derivatives along each axis (zero where the clamp is active).
template <int NDIM>
__device__ __forceinline__ void interp_grad(const Geom& g, const Feet<NDIM>& F, const float* f,
                                            float* val, float* dv) {
    const float* p = f + F.base;
    if constexpr (NDIM == 2) {
        const float fy = F.f[0].f, fx = F.f[1].f;
        const float c00 = p[0], c01 = p[1], c10 = p[g.P], c11 = p[g.P + 1];
        const float a = (1.f - fx) * c00 + fx * c01;
        const float b = (1.f - fx) * c10 + fx * c11;
        *val = (1.f - fy) * a + fy * b;
        dv[0] = F.f[0].inside ? (b - a) : 0.f;
        dv[1] = F.f[1].inside ? ((1.f - fy) * (c01 - c00) + fy * (c11 - c10)) : 0.f;
    } else {
        const float fz = F.f[0].f, fy = F.f[1].f, fx = F.f[2].f;
        const long long S = g.slab, P = g.P;
        const float c000 = p[0], c001 = p[1], c010 = p[P], c011 = p[P + 1];
        const float c100 = p[S], c101 = p[S + 1], c110 = p[S + P], c111 = p[S + P + 1];
        const float a0 = (1.f - fx) * c000 + fx * c001;
        const float a1 = (1.f - fx) * c010 + fx * c011;
        const float a2 = (1.f - fx) * c100 + fx * c101;
        const float a3 = (1.f - fx) * c110 + fx * c111;
        const float b0 = (1.f - fy) * a0 + fy * a1;
        const float b1 = (1.f - fy) * a2 + fy * a3;
        *val = (1.f - fz) * b0 + fz * b1;
        dv[0] = F.f[0].inside ? (b1 - b0) : 0.f;
        dv[1] = F.f[1].inside ? ((1.f - fz) * (a1 - a0) + fz * (a3 - a2)) : 0.f;
        const float e0 = (1.f - fy) * (c001 - c000) + fy * (c011 - c010);
        const float e1 = (1.f - fy) * (c101 - c100) + fy * (c111 - c110);
        dv[2] = F.f[2].inside ? ((1.f - fz) * e0 + fz * e1) : 0.f;
    }
}

template <int NDIM>
__device__ __forceinline__ void axis_info(const Geom& g, const Vox& v, int* c, int* n,
                                          long long* s) {
    if constexpr (NDIM == 2) {
        c[0] = v.y; n[0] = g.ny; s[0] = g.P;
        c[1] = v.x; n[1] = g.nx; s[1] = 1;
    } else {
        c[0] = v.z; n[0] = g.nz; s[0] = g.slab;
        c[1] = v.y; n[1] = g.ny; s[1] = g.P;
        c[2] = v.x; n[2] = g.nx; s[2] = 1;
    }
}

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
k_advect2d(Geom g, Coefs cf, int t, float* __restrict__ states, const float* __restrict__ u,
           unsigned int* __restrict__ maxdisp) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    constexpr int W = kPX + 2 * kAdvHalo;        // 40
    constexpr int HU = kPY + 2;                  // 10
    constexpr int HI = kPY + 2 * kAdvHalo;       // 16
    __shared__ __align__(16) float sU0[HU * W], sU1[HU * W], sI[HI * W], sP[HI * W];
    const int b = blockIdx.z;
    const int x0 = blockIdx.x * kPX, y0 = blockIdx.y * kPY;
    const float* u0 = slice_of(u, g, ((long long)t * 2 + 0) * g.B + b);
    const float* u1 = slice_of(u, g, ((long long)t * 2 + 1) * g.B + b);
    const float* It = slice_of(states, g, ((long long)t * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)t * 2 + 1) * g.B + b);
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
        float* I1 = slice_of(states, g, ((long long)(t + 1) * 2 + 0) * g.B + b);
        float* p1 = slice_of(states, g, ((long long)(t + 1) * 2 + 1) * g.B + b);
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
k_advect(Geom g, Coefs cf, int t, float* __restrict__ states, const float* __restrict__ u,
         unsigned int* __restrict__ maxdisp) {
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
            const float* ua = slice_of(u, g, ((long long)t * NDIM + a) * g.B + b);
            d[a] = disp_of(dtrho, ua[o]);
            du += cdiff(ua, o, s[a], c[a], n[a]);
            dmax = fmaxf(dmax, fabsf(d[a]));
        }
        const float div = -rho * du;  // div v, v = -rho u
        const Feet<NDIM> F = feet_of<NDIM>(g, v, d);
        const float* It = slice_of(states, g, ((long long)t * 2 + 0) * g.B + b);
        const float* pt = slice_of(states, g, ((long long)t * 2 + 1) * g.B + b);
        const float Iw = interp<NDIM>(g, F, It);
        const float pw = interp<NDIM>(g, F, pt);
        float* I1 = slice_of(states, g, ((long long)(t + 1) * 2 + 0) * g.B + b);
        float* p1 = slice_of(states, g, ((long long)(t + 1) * 2 + 1) * g.B + b);
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

// Cost partials: one CTA = 256 threads over a fixed voxel range of instance
// blockIdx.y; also writes the adjoint start I^_T = I_T - J, p^_T = 0.
template <int NDIM>
__global__ void __launch_bounds__(256)
k_cost_partials(Geom g, int T, const float* __restrict__ states, const float* __restrict__ u,
                const float* __restrict__ J, float* Ih, float* ph, float* Ihp, float* php,
                double* partials) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    const int b = blockIdx.y;
    const long long N = (long long)g.nz * g.ny * g.nx;
    const float* IT = slice_of(states, g, ((long long)T * 2 + 0) * g.B + b);
    const float* I0 = slice_of(states, g, (0LL * 2 + 0) * g.B + b);
    const float* p0 = slice_of(states, g, (0LL * 2 + 1) * g.B + b);
    double data = 0.0, kin = 0.0, res = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        Vox v;
        v.b = b;
        v.x = (int)(i % g.nx);
        v.y = (int)((i / g.nx) % g.ny);
        v.z = (int)(i / ((long long)g.nx * g.ny));
        const long long o = gidx(g, v.z, v.y, v.x);
        const float r = IT[o] - J[(long long)b * N + i];
        data += 0.5 * (double)r * (double)r;
        int c[NDIM], n[NDIM];
        long long s[NDIM];
        axis_info<NDIM>(g, v, c, n, s);
        const float p = p0[o];
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const float ga = cdiff(I0, o, s[a], c[a], n[a]);
            const float* ua = slice_of(u, g, (0LL * NDIM + a) * g.B + b);
            kin += (double)(p * ga) * (double)ua[o];
        }
        res += (double)p * (double)p;
        slice_of(Ih, g, b)[o] = r;
        slice_of(ph, g, b)[o] = 0.f;
        slice_of(Ihp, g, b)[o] = 0.f;  // scatter accumulators start at zero
        slice_of(php, g, b)[o] = 0.f;
    }
    __shared__ double red[3][256];
    red[0][threadIdx.x] = data;
    red[1][threadIdx.x] = kin;
    red[2][threadIdx.x] = res;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3)
        partials[((long long)b * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(256)
k_cost_final(int nblk, Coefs cf, const double* __restrict__ partials, double* cost) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    const int b = blockIdx.x;
    __shared__ double red[3][256];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nblk; i += blockDim.x)
        for (int k = 0; k < 3; ++k) acc[k] += partials[((long long)b * nblk + i) * 3 + k];
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double lam = (double)cf.lambda[b], rho = (double)cf.rho[b];
        cost[b * 3 + 0] = red[0][0];
        cost[b * 3 + 1] = lam * red[1][0];
        cost[b * 3 + 2] = lam * rho * red[2][0];
    }
}

template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_init(Geom g, const float* __restrict__ gI1, const float* __restrict__ gp1, float* Ih,
           float* ph, float* Ihp, float* php) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const long long o = (long long)v.b * g.inst + gidx(g, v.z, v.y, v.x);
    const long long ci = cidx(g, v);
    Ih[o] = gI1[ci];
    ph[o] = gp1 ? gp1[ci] : 0.f;
    Ihp[o] = 0.f;  // scatter accumulators start at zero
    php[o] = 0.f;
}

// Window radius of the gather-form transpose at step t: a source x feeds node
// n only if n lies in the cell of its foot, so |n - x| <= 1 + |d| per axis and
// R = 1 + floor(max |d|) bounds every contributing source.
__device__ __forceinline__ int gather_radius(const unsigned int* maxdisp, int t, int B, int b) {
    return 1 + (int)floorf(__uint_as_float(maxdisp[kMaxdispStride * ((long long)t * B + b)]));
}

template <int NDIM>
struct GatherTile;  // node tile of the gather kernel (256 nodes per CTA)
template <>
struct GatherTile<2> {
    static constexpr int TX = 32, TY = 8, TZ = 1, RMAX = 8;
};
template <>
struct GatherTile<3> {
    static constexpr int TX = 8, TY = 8, TZ = 4, RMAX = 2;
};

template <int NDIM>
__host__ __device__ constexpr int gather_region() {
    using G = GatherTile<NDIM>;
    return (G::TX + 2 * G::RMAX) * (G::TY + 2 * G::RMAX) *
           (NDIM == 3 ? (G::TZ + 2 * G::RMAX) : 1);
}

template <int NDIM>
dim3 gather_grid(const Geom& g) {
    using G = GatherTile<NDIM>;
    return dim3((g.nx + G::TX - 1) / G::TX,
                ((g.ny + G::TY - 1) / G::TY) * ((g.nz + G::TZ - 1) / G::TZ), g.B);
}

// Packs the foot cell of a source relative to the source: one byte per axis
// (offset + 64), bit 24 + a when the clamp on axis a is inactive, bit 31 for
// sources outside the domain.
__device__ __forceinline__ int pack_cell(const int* off, const bool* inside) {
    return (off[0] + 64) | ((off[1] + 64) << 8) | ((off[2] + 64) << 16) |
           (inside[0] ? (1 << 24) : 0) | (inside[1] ? (1 << 25) : 0) |
           (inside[2] ? (1 << 26) : 0);
}
__device__ __forceinline__ int cell_off(int cell, int a) { return ((cell >> (8 * a)) & 0xff) - 64; }

// S^T at one node by gather over the staged foot records of its window
// (2R+1)^d, in a fixed order: node - source - cell offset must be 0 or 1 on
// every axis.  Records are indexed ((z * RY) + y) * RX + x in the staged region.
template <int NDIM>
__device__ __forceinline__ void gather_window(const int* s_cell, const float* const* s_f,
                                              const float* s_I, const float* s_P, int RX, int RY,
                                              int lx, int ly, int lz, int R, float* accI,
                                              float* accP) {
    float aI = 0.f, aP = 0.f;
    for (int dz = (NDIM == 3 ? -R : 0); dz <= (NDIM == 3 ? R : 0); ++dz) {
        for (int dy = -R; dy <= R; ++dy) {
            const int rowbase = ((lz + dz) * RY + (ly + dy)) * RX + lx;
            for (int dx = -R; dx <= R; ++dx) {
                const int i = rowbase + dx;
                const int cell = s_cell[i];
                const int ex = -dx - cell_off(cell, NDIM - 1);
                const int ey = -dy - cell_off(cell, NDIM - 2);
                const int ez = (NDIM == 3) ? -dz - cell_off(cell, 0) : 0;
                if (cell < 0 || (unsigned)ex > 1u || (unsigned)ey > 1u || (unsigned)ez > 1u)
                    continue;
                float w;
                if constexpr (NDIM == 2) {
                    const float fy = s_f[0][i], fx = s_f[1][i];
                    w = (ey ? fy : 1.f - fy) * (ex ? fx : 1.f - fx);
                } else {
                    const float fz = s_f[0][i], fy = s_f[1][i], fx = s_f[2][i];
                    w = (ez ? fz : 1.f - fz) * (ey ? fy : 1.f - fy) * (ex ? fx : 1.f - fx);
                }
                aI += w * s_I[i];
                aP += w * s_P[i];
            }
        }
    }
    *accI = aI;
    *accP = aP;
}

template <int NDIM>
__host__ __device__ constexpr int transport_smem_words() {
    // general path: cell, f[NDIM], I, P, D records over the RMAX region;
    // 2-D fast path: records over tile (+) 2 and six staged windows.
    return NDIM == 2 ? ((1 + 2 + 3) * gather_region<2>() > 6400 ? (1 + 2 + 3) * gather_region<2>()
                                                                 : 6400)
                     : (1 + 3 + 3) * gather_region<3>();
}

constexpr int kFastH2 = 2;  // 2-D fast path: per-step displacement < 2 voxels

// 2-D adjoint step for instances whose per-step displacement is below
// H <= kFastH2 voxels: u, I_t, p_t, I^' and p^' are staged asynchronously over
// the tile grown by the halos the step needs (u: H+1, I_t/p_t: 2H+1, I^'/p^': H),
// and every stencil, interpolation and gather then reads shared memory.
template <int H>
__device__ __forceinline__ void transport_fast2d(const Geom& g, float rho, float mu, float dt,
                                                 const float* It, const float* pt,
                                                 const float* u0, const float* u1,
                                                 const float* Ihb, const float* phb, float* vh0,
                                                 float* vh1, float* Ihpb, float* phpb,
                                                 float* smem, unsigned int* s_dmax) {
    using G = GatherTile<2>;
    constexpr int WU = G::TX + 8, WI = G::TX + 16, WA = G::TX + 8;
    constexpr int HU = G::TY + 2 * H + 2, HI = G::TY + 4 * H + 2, HA = G::TY + 2 * H;
    constexpr int RX = G::TX + 2 * H, RY = G::TY + 2 * H, NR = RX * RY;
    const float dtrho = dt * rho;
    const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * G::TY;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kPX + tx;
    int* s_cell = reinterpret_cast<int*>(smem);
    float* s_f0 = smem + NR;
    float* s_f1 = s_f0 + NR;
    float* s_I = s_f1 + NR;
    float* s_P = s_I + NR;
    float* s_D = s_P + NR;
    float* sU0 = s_D + NR;   // 16-byte aligned: NR * 6 words is a multiple of 4
    float* sU1 = sU0 + WU * HU;
    float* sI = sU1 + WU * HU;
    float* sP = sI + WI * HI;
    float* sIh = sP + WI * HI;
    float* sPh = sIh + WA * HA;
    const int xu = x0 - 4, yu = y0 - H - 1;
    const int xi = x0 - 8, yi = y0 - 2 * H - 1;
    const int xa = x0 - 4, ya = y0 - H;
    stage_async<WU, HU>(sU0, u0, g, xu, yu);
    stage_async<WU, HU>(sU1, u1, g, xu, yu);
    stage_async<WI, HI>(sI, It, g, xi, yi);
    stage_async<WI, HI>(sP, pt, g, xi, yi);
    stage_async<WA, HA>(sIh, Ihb, g, xa, ya);
    stage_async<WA, HA>(sPh, phb, g, xa, ya);
    cp_async_wait_all();
    __syncthreads();

    // Phase 1: records of the sources of tile (+) H.
    float dmax = 0.f;
    for (int i = tid; i < NR; i += kPX * kPY) {
        const int ry = i / RX, rx = i - ry * RX;
        const int sx = x0 - H + rx, sy = y0 - H + ry;
        int cell = (int)0x80000000;
        float f0 = 0.f, f1 = 0.f, fI = 0.f, fP = 0.f, fD = 0.f;
        if (sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny) {
            const int ui = (sy - yu) * WU + (sx - xu);
            const float d0 = disp_of(dtrho, sU0[ui]);
            const float d1 = disp_of(dtrho, sU1[ui]);
            dmax = fmaxf(dmax, fmaxf(fabsf(d0), fabsf(d1)));
            float du = 0.f;
            du += 0.5f * (sU0[ui + (sy < g.ny - 1 ? WU : 0)] - sU0[ui - (sy > 0 ? WU : 0)]);
            du += 0.5f * (sU1[ui + (sx < g.nx - 1 ? 1 : 0)] - sU1[ui - (sx > 0 ? 1 : 0)]);
            const float div = -rho * du;
            const Foot1 fy = foot1(sy, d0, g.ny), fx = foot1(sx, d1, g.nx);
            const float pw = bilin(sP + (fy.i0 - yi) * WI + (fx.i0 - xi), WI, fy.f, fx.f);
            const int ai = (sy - ya) * WA + (sx - xa);
            const float phv = sPh[ai];
            fI = sIh[ai];
            fP = phv * (1.f - dt * div) + (dt * mu) * fI;
            fD = -dt * pw * phv;
            const int off[3] = {fy.i0 - sy, fx.i0 - sx, 0};
            const bool ins[3] = {fy.inside, fx.inside, false};
            cell = pack_cell(off, ins);
            f0 = fy.f;
            f1 = fx.f;
        }
        s_cell[i] = cell;
        s_f0[i] = f0;
        s_f1[i] = f1;
        s_I[i] = fI;
        s_P[i] = fP;
        s_D[i] = fD;
    }
    const unsigned int wmax = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
    if ((tx & 31) == 0 && wmax) atomicMax(s_dmax, wmax);
    __syncthreads();

    const int x = x0 + tx, y = y0 + ty;
    if (x >= g.nx || y >= g.ny) return;
    const int me = (ty + H) * RX + tx + H;
    const int R = 1 + (int)floorf(__uint_as_float(*s_dmax));
    const float* fptr[2] = {s_f0, s_f1};
    float accI, accP;
    gather_window<2>(s_cell, fptr, s_I, s_P, RX, RY, tx + H, ty + H, 0, R, &accI, &accP);
    const int o = y * g.P + x;
    Ihpb[o] = accI;
    phpb[o] = accP;

    // y^ from this node's own foot, v^ = -dt y^ + D^T div^.
    const int cell = s_cell[me];
    const int iy = y + cell_off(cell, 0), ix = x + cell_off(cell, 1);
    const float fy = s_f0[me], fx = s_f1[me];
    const bool iny = (cell >> 24) & 1, inx = (cell >> 25) & 1;
    const int ci = (iy - yi) * WI + (ix - xi);
    float dIy, dIx, dPy, dPx;
    bilin_grad(sI + ci, WI, fy, fx, iny, inx, &dIy, &dIx);
    bilin_grad(sP + ci, WI, fy, fx, iny, inx, &dPy, &dPx);
    const float Ihv = s_I[me], pthv = s_P[me];
    float dT0 = 0.f, dT1 = 0.f;
    if (y >= 1) dT0 += 0.5f * s_D[me - RX];
    if (y == g.ny - 1) dT0 += 0.5f * s_D[me];
    if (y <= g.ny - 2) dT0 -= 0.5f * s_D[me + RX];
    if (y == 0) dT0 -= 0.5f * s_D[me];
    if (x >= 1) dT1 += 0.5f * s_D[me - 1];
    if (x == g.nx - 1) dT1 += 0.5f * s_D[me];
    if (x <= g.nx - 2) dT1 -= 0.5f * s_D[me + 1];
    if (x == 0) dT1 -= 0.5f * s_D[me];
    vh0[o] = -dt * (dIy * Ihv + dPy * pthv) + dT0;
    vh1[o] = -dt * (dIx * Ihv + dPx * pthv) + dT1;
}

// Per-axis weights with which a source passes its value to the nodes s-1, s,
// s+1 when its foot moved by less than one voxel: the cell offset is -1 or 0,
// so the two non-zero corner weights land on (s-1, s) or (s, s+1).
__device__ __forceinline__ void axis_weights(const Foot1& f, int s, float* w) {
    const bool down = (f.i0 - s) < 0;
    w[0] = down ? 1.f - f.f : 0.f;
    w[1] = down ? f.f : 1.f - f.f;
    w[2] = down ? 0.f : f.f;
}

// 2-D adjoint step for instances whose per-step displacement is below one
// voxel (H = R = 1).  Same staging as transport_fast2d<1>; the window becomes
// nine branch-free products of per-axis weights (zero weights add exact
// zeros, so sums equal the record-based gather's).
__device__ __forceinline__ void transport_r1_2d(const Geom& g, float rho, float mu, float dt,
                                                const float* It, const float* pt,
                                                const float* u0, const float* u1,
                                                const float* Ihb, const float* phb, float* vh0,
                                                float* vh1, float* Ihpb, float* phpb,
                                                float* smem) {
    using G = GatherTile<2>;
    constexpr int H = 1;
    constexpr int WU = G::TX + 8, WI = G::TX + 16, WA = G::TX + 8;
    constexpr int HU = G::TY + 2 * H + 2, HI = G::TY + 4 * H + 2, HA = G::TY + 2 * H;
    constexpr int RX = G::TX + 2 * H, RY = G::TY + 2 * H, NR = RX * RY;
    const float dtrho = dt * rho;
    const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * G::TY;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kPX + tx;
    float* sWy = smem;             // [3][NR]
    float* sWx = sWy + 3 * NR;     // [3][NR]
    float* s_I = sWx + 3 * NR;
    float* s_P = s_I + NR;
    float* s_D = s_P + NR;
    float* sU0 = s_D + NR;         // 9 * NR = 3060 words: 16-byte aligned
    float* sU1 = sU0 + WU * HU;
    float* sI = sU1 + WU * HU;
    float* sP = sI + WI * HI;
    float* sIh = sP + WI * HI;
    float* sPh = sIh + WA * HA;
    const int xu = x0 - 4, yu = y0 - H - 1;
    const int xi = x0 - 8, yi = y0 - 2 * H - 1;
    const int xa = x0 - 4, ya = y0 - H;
    stage_async<WU, HU>(sU0, u0, g, xu, yu);
    stage_async<WU, HU>(sU1, u1, g, xu, yu);
    stage_async<WI, HI>(sI, It, g, xi, yi);
    stage_async<WI, HI>(sP, pt, g, xi, yi);
    stage_async<WA, HA>(sIh, Ihb, g, xa, ya);
    stage_async<WA, HA>(sPh, phb, g, xa, ya);
    cp_async_wait_all();
    __syncthreads();

    // Phase 1: per-axis weights, I^', p~^ and div^ of the sources of tile (+) 1.
    for (int i = tid; i < NR; i += kPX * kPY) {
        const int ry = i / RX, rx = i - ry * RX;
        const int sx = x0 - H + rx, sy = y0 - H + ry;
        float wy[3] = {0.f, 0.f, 0.f}, wx[3] = {0.f, 0.f, 0.f};
        float fI = 0.f, fP = 0.f, fD = 0.f;
        if (sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny) {
            const int ui = (sy - yu) * WU + (sx - xu);
            const float d0 = disp_of(dtrho, sU0[ui]);
            const float d1 = disp_of(dtrho, sU1[ui]);
            float du = 0.f;
            du += 0.5f * (sU0[ui + (sy < g.ny - 1 ? WU : 0)] - sU0[ui - (sy > 0 ? WU : 0)]);
            du += 0.5f * (sU1[ui + (sx < g.nx - 1 ? 1 : 0)] - sU1[ui - (sx > 0 ? 1 : 0)]);
            const float div = -rho * du;
            const Foot1 fy = foot1(sy, d0, g.ny), fx = foot1(sx, d1, g.nx);
            const float pw = bilin(sP + (fy.i0 - yi) * WI + (fx.i0 - xi), WI, fy.f, fx.f);
            const int ai = (sy - ya) * WA + (sx - xa);
            const float phv = sPh[ai];
            fI = sIh[ai];
            fP = phv * (1.f - dt * div) + (dt * mu) * fI;
            fD = -dt * pw * phv;
            axis_weights(fy, sy, wy);
            axis_weights(fx, sx, wx);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sWy[k * NR + i] = wy[k];
            sWx[k * NR + i] = wx[k];
        }
        s_I[i] = fI;
        s_P[i] = fP;
        s_D[i] = fD;
    }
    __syncthreads();

    const int x = x0 + tx, y = y0 + ty;
    if (x >= g.nx || y >= g.ny) return;
    const int me = (ty + H) * RX + tx + H;
    // Phase 2a: S^T, sources at (dy, dx) in {-1,0,1}^2 pass weight
    // wy[1 - dy] * wx[1 - dx] to this node.
    float accI = 0.f, accP = 0.f;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int i = me + dy * RX + dx;
            const float w = sWy[(1 - dy) * NR + i] * sWx[(1 - dx) * NR + i];
            accI += w * s_I[i];
            accP += w * s_P[i];
        }
    }
    const int o = y * g.P + x;
    Ihpb[o] = accI;
    phpb[o] = accP;

    // Phase 2b: y^ from this node's own foot (recomputed from the staged u).
    const int ui = (y - yu) * WU + (x - xu);
    const Foot1 fy = foot1(y, disp_of(dtrho, sU0[ui]), g.ny);
    const Foot1 fx = foot1(x, disp_of(dtrho, sU1[ui]), g.nx);
    const int ci = (fy.i0 - yi) * WI + (fx.i0 - xi);
    float dIy, dIx, dPy, dPx;
    bilin_grad(sI + ci, WI, fy.f, fx.f, fy.inside, fx.inside, &dIy, &dIx);
    bilin_grad(sP + ci, WI, fy.f, fx.f, fy.inside, fx.inside, &dPy, &dPx);
    const float Ihv = s_I[me], pthv = s_P[me];
    float dT0 = 0.f, dT1 = 0.f;
    if (y >= 1) dT0 += 0.5f * s_D[me - RX];
    if (y == g.ny - 1) dT0 += 0.5f * s_D[me];
    if (y <= g.ny - 2) dT0 -= 0.5f * s_D[me + RX];
    if (y == 0) dT0 -= 0.5f * s_D[me];
    if (x >= 1) dT1 += 0.5f * s_D[me - 1];
    if (x == g.nx - 1) dT1 += 0.5f * s_D[me];
    if (x <= g.nx - 2) dT1 -= 0.5f * s_D[me + 1];
    if (x == 0) dT1 -= 0.5f * s_D[me];
    vh0[o] = -dt * (dIy * Ihv + dPy * pthv) + dT0;
    vh1[o] = -dt * (dIx * Ihv + dPx * pthv) + dT1;
}

// 3-D adjoint step for instances whose per-step displacement is below one
// voxel (R = 1): per-axis weight records of the sources of tile (+) 1 in shared
// memory, a branch-free 27-candidate window, operands read through L1 with
// 32-bit offsets inside the instance.  Same expressions as the general path.
__device__ __forceinline__ void transport_r1_3d(const Geom& g, float rho, float mu, float dt,
                                                const float* It, const float* pt,
                                                const float* u0, const float* u1,
                                                const float* u2, const float* Ihb,
                                                const float* phb, float* vh0, float* vh1,
                                                float* vh2, float* Ihpb, float* phpb,
                                                float* smem) {
    using G = GatherTile<3>;
    constexpr int RX = G::TX + 2, RY = G::TY + 2, RZ = G::TZ + 2, NR = RX * RY * RZ;
    const float dtrho = dt * rho;
    const int tid = threadIdx.y * kPX + threadIdx.x;
    const int nty = (g.ny + G::TY - 1) / G::TY;
    const int x0 = blockIdx.x * G::TX;
    const int y0 = (blockIdx.y % nty) * G::TY;
    const int z0 = (blockIdx.y / nty) * G::TZ;
    const int P = g.P, S = (int)g.slab;
    float* sW = smem;          // [9][NR]: wz[3], wy[3], wx[3]
    float* s_I = sW + 9 * NR;
    float* s_P = s_I + NR;
    float* s_D = s_P + NR;

    for (int i = tid; i < NR; i += kPX * kPY) {
        const int rz = i / (RX * RY), ry = (i / RX) % RY, rx = i % RX;
        const int sx = x0 - 1 + rx, sy = y0 - 1 + ry, sz = z0 - 1 + rz;
        float w[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float fI = 0.f, fP = 0.f, fD = 0.f;
        if (sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz) {
            const int o = sz * S + sy * P + sx;
            const float a0 = __ldg(u0 + o), a1 = __ldg(u1 + o), a2 = __ldg(u2 + o);
            const float d0 = disp_of(dtrho, a0), d1 = disp_of(dtrho, a1), d2 = disp_of(dtrho, a2);
            float du = 0.f;
            du += 0.5f * (__ldg(u0 + o + (sz < g.nz - 1 ? S : 0)) - __ldg(u0 + o - (sz > 0 ? S : 0)));
            du += 0.5f * (__ldg(u1 + o + (sy < g.ny - 1 ? P : 0)) - __ldg(u1 + o - (sy > 0 ? P : 0)));
            du += 0.5f * (__ldg(u2 + o + (sx < g.nx - 1 ? 1 : 0)) - __ldg(u2 + o - (sx > 0 ? 1 : 0)));
            const float div = -rho * du;
            const Foot1 fz = foot1(sz, d0, g.nz), fy = foot1(sy, d1, g.ny), fx = foot1(sx, d2, g.nx);
            const float* q = pt + (fz.i0 * S + fy.i0 * P + fx.i0);
            const float c0 = (1.f - fx.f) * __ldg(q) + fx.f * __ldg(q + 1);
            const float c1 = (1.f - fx.f) * __ldg(q + P) + fx.f * __ldg(q + P + 1);
            const float c2 = (1.f - fx.f) * __ldg(q + S) + fx.f * __ldg(q + S + 1);
            const float c3 = (1.f - fx.f) * __ldg(q + S + P) + fx.f * __ldg(q + S + P + 1);
            const float b0 = (1.f - fy.f) * c0 + fy.f * c1;
            const float b1 = (1.f - fy.f) * c2 + fy.f * c3;
            const float pw = (1.f - fz.f) * b0 + fz.f * b1;
            const float phv = __ldg(phb + o);
            fI = __ldg(Ihb + o);
            fP = phv * (1.f - dt * div) + (dt * mu) * fI;
            fD = -dt * pw * phv;
            axis_weights(fz, sz, w);
            axis_weights(fy, sy, w + 3);
            axis_weights(fx, sx, w + 6);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) sW[k * NR + i] = w[k];
        s_I[i] = fI;
        s_P[i] = fP;
        s_D[i] = fD;
    }
    __syncthreads();

    const int x = x0 + (tid & 7), y = y0 + ((tid >> 3) & 7), z = z0 + (tid >> 6);
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    const int me = ((z - z0 + 1) * RY + (y - y0 + 1)) * RX + (x - x0 + 1);
    float accI = 0.f, accP = 0.f;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int i = me + (dz * RY + dy) * RX + dx;
                const float w = (sW[(1 - dz) * NR + i] * sW[(4 - dy) * NR + i]) *
                                sW[(7 - dx) * NR + i];
                accI += w * s_I[i];
                accP += w * s_P[i];
            }
        }
    }
    const int o = z * S + y * P + x;
    Ihpb[o] = accI;
    phpb[o] = accP;

    // y^ from this node's own foot, v^ = -dt y^ + D^T div^.
    const Foot1 fz = foot1(z, disp_of(dtrho, __ldg(u0 + o)), g.nz);
    const Foot1 fy = foot1(y, disp_of(dtrho, __ldg(u1 + o)), g.ny);
    const Foot1 fx = foot1(x, disp_of(dtrho, __ldg(u2 + o)), g.nx);
    const int cb = fz.i0 * S + fy.i0 * P + fx.i0;
    float dI[3], dP[3];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        const float* q = (f == 0 ? It : pt) + cb;
        const float c000 = __ldg(q), c001 = __ldg(q + 1), c010 = __ldg(q + P), c011 = __ldg(q + P + 1);
        const float c100 = __ldg(q + S), c101 = __ldg(q + S + 1), c110 = __ldg(q + S + P),
                    c111 = __ldg(q + S + P + 1);
        const float a0 = (1.f - fx.f) * c000 + fx.f * c001;
        const float a1 = (1.f - fx.f) * c010 + fx.f * c011;
        const float a2 = (1.f - fx.f) * c100 + fx.f * c101;
        const float a3 = (1.f - fx.f) * c110 + fx.f * c111;
        const float b0 = (1.f - fy.f) * a0 + fy.f * a1;
        const float b1 = (1.f - fy.f) * a2 + fy.f * a3;
        float* dv = f == 0 ? dI : dP;
        dv[0] = fz.inside ? (b1 - b0) : 0.f;
        dv[1] = fy.inside ? ((1.f - fz.f) * (a1 - a0) + fz.f * (a3 - a2)) : 0.f;
        const float e0 = (1.f - fy.f) * (c001 - c000) + fy.f * (c011 - c010);
        const float e1 = (1.f - fy.f) * (c101 - c100) + fy.f * (c111 - c110);
        dv[2] = fx.inside ? ((1.f - fz.f) * e0 + fz.f * e1) : 0.f;
    }
    const float Ihv = s_I[me], pthv = s_P[me];
    const int rs[3] = {RX * RY, RX, 1};
    const int cc[3] = {z, y, x}, nn[3] = {g.nz, g.ny, g.nx};
    float* vhs[3] = {vh0, vh1, vh2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float dT = 0.f;
        if (cc[a] >= 1) dT += 0.5f * s_D[me - rs[a]];
        if (cc[a] == nn[a] - 1) dT += 0.5f * s_D[me];
        if (cc[a] <= nn[a] - 2) dT -= 0.5f * s_D[me + rs[a]];
        if (cc[a] == 0) dT -= 0.5f * s_D[me];
        vhs[a][o] = -dt * (dI[a] * Ihv + dP[a] * pthv) + dT;
    }
}

// One adjoint step t, fused: for every source of the node tile grown by a halo
// H it forms p~^ = p^'(1 - dt div v) + dt mu I^' and div^ = -dt p~ p^' and the
// foot record, then for every node of the tile
//   I^ (partial) = S^T I^',  p^ (partial) = S^T p~^      (gather, fixed order)
//   v^_a = -dt y^_a + D_a^T div^,  y^_a = d(interp I_t)/dy_a I^' + d(interp p_t)/dy_a p~^.
// Gather mode (R <= RMAX): H = R and the window of each node is the tile's own
// R_tile = 1 + floor(max |d| over the staged sources) <= R.  Scatter mode
// (R > RMAX): H = 1 and each CTA scatters S^T of its own sources into Ihp / php
// with atomics (bounded work; k_adj_gradp reads them after the launch).
// 2-D instances with R <= kFastH2 take transport_fast2d.
template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_transport(Geom g, Coefs cf, int t, const float* __restrict__ states,
                const float* __restrict__ u, const unsigned int* __restrict__ maxdisp,
                const float* __restrict__ Ih1, const float* __restrict__ ph1, float* vh,
                float* Ihp, float* php, unsigned int* fault) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    using G = GatherTile<NDIM>;
    constexpr int REG = gather_region<NDIM>();
    __shared__ __align__(16) float smem[transport_smem_words<NDIM>()];
    __shared__ unsigned int s_dmax;

    const int b = blockIdx.z;
    const float rho = cf.rho[b], mu = cf.mu[b], dt = cf.dt;
    const float dtrho = dt * rho;
    const int tid = threadIdx.y * kPX + threadIdx.x;
    const float* ub[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) ub[a] = slice_of(u, g, ((long long)t * NDIM + a) * g.B + b);
    const float* It = slice_of(states, g, ((long long)t * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)t * 2 + 1) * g.B + b);
    const float* Ihb = Ih1 + (long long)b * g.inst;
    const float* phb = ph1 + (long long)b * g.inst;
    float* Isc = Ihp + (long long)b * g.inst;
    float* Psc = php + (long long)b * g.inst;
    const int Rinst = gather_radius(maxdisp, t, g.B, b);
    if (tid == 0) s_dmax = 0u;
    if constexpr (NDIM == 3) {
        if (Rinst == 1) {
            __syncthreads();
            transport_r1_3d(g, rho, mu, dt, It, pt, ub[0], ub[1], ub[2], Ihb, phb,
                            vh + (long long)b * g.inst, vh + ((long long)g.B + b) * g.inst,
                            vh + (2LL * g.B + b) * g.inst, Isc, Psc, smem);
            return;
        }
    }
    if constexpr (NDIM == 2) {
        if (Rinst <= kFastH2) {
            __syncthreads();
            float* vh0 = vh + (long long)b * g.inst;
            float* vh1 = vh + ((long long)g.B + b) * g.inst;
            if (Rinst == 1)
                transport_r1_2d(g, rho, mu, dt, It, pt, ub[0], ub[1], Ihb, phb, vh0, vh1, Isc,
                                Psc, smem);
            else
                transport_fast2d<2>(g, rho, mu, dt, It, pt, ub[0], ub[1], Ihb, phb, vh0, vh1, Isc,
                                    Psc, smem, &s_dmax);
            return;
        }
    }
    int* s_cell = reinterpret_cast<int*>(smem);
    const float* s_fc[NDIM];
    float* s_f[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) s_fc[a] = s_f[a] = smem + (1 + a) * REG;
    float* s_I = smem + (1 + NDIM) * REG;   // I^' of the source
    float* s_P = s_I + REG;                 // p~^ of the source
    float* s_D = s_P + REG;                 // div^ of the source

    const int nty = (g.ny + G::TY - 1) / G::TY;
    const int x0 = blockIdx.x * G::TX;
    const int y0 = (blockIdx.y % nty) * G::TY;
    const int z0 = (blockIdx.y / nty) * G::TZ;
    Vox v;
    v.b = b;
    if constexpr (NDIM == 2) {
        v.x = x0 + threadIdx.x;
        v.y = y0 + threadIdx.y;
        v.z = 0;
    } else {
        v.x = x0 + (tid & 7);
        v.y = y0 + ((tid >> 3) & 7);
        v.z = z0 + (tid >> 6);
    }
    v.ok = v.x < g.nx && v.y < g.ny && v.z < g.nz;
    const bool gather = Rinst <= G::RMAX;  // uniform over the CTA
    const int H = gather ? Rinst : 1;
    const int RX = G::TX + 2 * H, RY = G::TY + 2 * H;
    const int RZ = (NDIM == 3) ? G::TZ + 2 * H : 1;
    const int nreg = RX * RY * RZ;
    __syncthreads();

    // Phase 1: per staged source.
    float dmax = 0.f;
    bool scattered = false;
    for (int i = tid; i < nreg; i += kPX * kPY) {
        const int rx = i % RX;
        const int ry = (i / RX) % RY;
        const int rz = i / (RX * RY);
        Vox sv;
        sv.b = b;
        sv.x = x0 - H + rx;
        sv.y = y0 - H + ry;
        sv.z = (NDIM == 3) ? z0 - H + rz : 0;
        int cell = (int)0x80000000;
        float ff[NDIM], fI = 0.f, fP = 0.f, fD = 0.f;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) ff[a] = 0.f;
        if (sv.x >= 0 && sv.x < g.nx && sv.y >= 0 && sv.y < g.ny && sv.z >= 0 && sv.z < g.nz) {
            const long long so = gidx(g, sv.z, sv.y, sv.x);
            int c[NDIM], n[NDIM];
            long long st[NDIM];
            axis_info<NDIM>(g, sv, c, n, st);
            float d[NDIM];
            float du = 0.f;
#pragma unroll
            for (int a = 0; a < NDIM; ++a) {
                d[a] = disp_of(dtrho, ub[a][so]);
                du += cdiff(ub[a], so, st[a], c[a], n[a]);
                dmax = fmaxf(dmax, fabsf(d[a]));
            }
            const float div = -rho * du;
            const Feet<NDIM> F = feet_of<NDIM>(g, sv, d);
            const float pw = interp<NDIM>(g, F, pt);
            const float phv = phb[so];
            fI = Ihb[so];
            fP = phv * (1.f - dt * div) + (dt * mu) * fI;
            fD = -dt * pw * phv;
            int off[3] = {0, 0, 0};
            bool ins[3] = {false, false, false};
#pragma unroll
            for (int a = 0; a < NDIM; ++a) {
                off[a] = F.f[a].i0 - c[a];
                ins[a] = F.f[a].inside;
                ff[a] = F.f[a].f;
            }
            cell = pack_cell(off, ins);
            const bool own = sv.x >= x0 && sv.x < x0 + G::TX && sv.y >= y0 && sv.y < y0 + G::TY &&
                             (NDIM == 2 || (sv.z >= z0 && sv.z < z0 + G::TZ));
            if (!gather && own) {
                // S^T by scatter: 2^d corners per source, order not fixed.
                scattered = true;
#pragma unroll
                for (int k = 0; k < (1 << NDIM); ++k) {
                    float w = 1.f;
                    long long q = F.base;
#pragma unroll
                    for (int a = 0; a < NDIM; ++a) {
                        const int up = (k >> a) & 1;
                        w *= up ? F.f[a].f : 1.f - F.f[a].f;
                        q += up ? st[a] : 0;
                    }
                    atomicAdd(Isc + q, w * fI);
                    atomicAdd(Psc + q, w * fP);
                }
            }
        }
        s_cell[i] = cell;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) s_f[a][i] = ff[a];
        s_I[i] = fI;
        s_P[i] = fP;
        s_D[i] = fD;
    }
    if (scattered) atomicOr(fault, kInfoScatter);
    const unsigned int wmax = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
    if ((tid & 31) == 0 && wmax) atomicMax(&s_dmax, wmax);
    __syncthreads();

    if (!v.ok) return;
    const int lx = v.x - x0 + H, ly = v.y - y0 + H;
    const int lz = (NDIM == 3) ? v.z - z0 + H : 0;
    const int me = (lz * RY + ly) * RX + lx;
    const long long o = gidx(g, v.z, v.y, v.x);
    const long long ob = (long long)b * g.inst + o;

    // Phase 2a: S^T by gather over the tile's window (fixed order, no atomics).
    if (gather) {
        const int R = 1 + (int)floorf(__uint_as_float(s_dmax));  // <= Rinst
        float accI, accP;
        gather_window<NDIM>(s_cell, s_fc, s_I, s_P, RX, RY, lx, ly, lz, R, &accI, &accP);
        Ihp[ob] = accI;
        php[ob] = accP;
    }

    // Phase 2b: foot derivative of this node's own backtracking, and v^.
    int c[NDIM], n[NDIM];
    long long st[NDIM];
    axis_info<NDIM>(g, v, c, n, st);
    const int cell = s_cell[me];
    Feet<NDIM> F;
    int i0[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        i0[a] = c[a] + cell_off(cell, a);
        F.f[a].i0 = i0[a];
        F.f[a].f = s_f[a][me];
        F.f[a].inside = (cell >> (24 + a)) & 1;
    }
    if constexpr (NDIM == 2)
        F.base = gidx(g, 0, i0[0], i0[1]);
    else
        F.base = gidx(g, i0[0], i0[1], i0[2]);
    float Iv, pv, dI[NDIM], dP[NDIM];
    interp_grad<NDIM>(g, F, It, &Iv, dI);
    interp_grad<NDIM>(g, F, pt, &pv, dP);
    const float Ihv = s_I[me], pthv = s_P[me];
    const int rstride[3] = {RX * RY, RX, 1};
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const int rs = (NDIM == 2) ? rstride[a + 1] : rstride[a];
        // (D_a^T div^) at this node from the staged neighbours
        float dT = 0.f;
        if (c[a] >= 1) dT += 0.5f * s_D[me - rs];
        if (c[a] == n[a] - 1) dT += 0.5f * s_D[me];
        if (c[a] <= n[a] - 2) dT -= 0.5f * s_D[me + rs];
        if (c[a] == 0) dT -= 0.5f * s_D[me];
        const float yh = dI[a] * Ihv + dP[a] * pthv;
        vh[((long long)a * g.B + b) * g.inst + o] = -dt * yh + dT;
    }
}

// 2-D k_adj_gradp on a 32 x 8 tile: m^ (both components), I_t and p_t staged
// with a one-voxel halo by cp.async; the same expressions as k_adj_gradp.
__global__ void __launch_bounds__(kPX * kPY)
k_adj_gradp2d(Geom g, Coefs cf, int t, int mode, const float* __restrict__ states,
              const float* __restrict__ u, const unsigned int* __restrict__ maxdisp,
              const float* __restrict__ mh, float* Ihp, float* php, float* Ih, float* ph,
              float* out0, float* gI0) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    constexpr int W = kPX + 8, HR = kPY + 2;
    __shared__ __align__(16) float sM0[HR * W], sM1[HR * W], sI[HR * W], sP[HR * W];
    const int b = blockIdx.z;
    const int x0 = blockIdx.x * kPX, y0 = blockIdx.y * kPY;
    const float* It = slice_of(states, g, ((long long)t * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)t * 2 + 1) * g.B + b);
    const float* m0 = mh + (long long)b * g.inst;
    const float* m1 = mh + ((long long)g.B + b) * g.inst;
    stage_async<W, HR>(sM0, m0, g, x0 - 4, y0 - 1);
    stage_async<W, HR>(sM1, m1, g, x0 - 4, y0 - 1);
    stage_async<W, HR>(sI, It, g, x0 - 4, y0 - 1);
    stage_async<W, HR>(sP, pt, g, x0 - 4, y0 - 1);
    cp_async_wait_all();
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= g.nx || y >= g.ny) return;
    const int o = y * g.P + x;
    const long long ob = (long long)b * g.inst + o;
    const int c = (threadIdx.y + 1) * W + threadIdx.x + 4;
    float phv = php[ob];
    float Ihv = Ihp[ob];
    if (t > 0 && gather_radius(maxdisp, t - 1, g.B, b) > GatherTile<2>::RMAX) {
        Ihp[ob] = 0.f;  // the next (earlier) step scatters into these
        php[ob] = 0.f;
    }
    // axis 0 (y): stride W in the staged tile
    const float g0 = 0.5f * (sI[c + (y < g.ny - 1 ? W : 0)] - sI[c - (y > 0 ? W : 0)]);
    phv += sM0[c] * g0;
    {
        float r = 0.f;
        if (y >= 1) r += 0.5f * (sM0[c - W] * sP[c - W]);
        if (y == g.ny - 1) r += 0.5f * (sM0[c] * sP[c]);
        if (y <= g.ny - 2) r -= 0.5f * (sM0[c + W] * sP[c + W]);
        if (y == 0) r -= 0.5f * (sM0[c] * sP[c]);
        Ihv += r;
    }
    // axis 1 (x)
    const float g1 = 0.5f * (sI[c + (x < g.nx - 1 ? 1 : 0)] - sI[c - (x > 0 ? 1 : 0)]);
    phv += sM1[c] * g1;
    {
        float r = 0.f;
        if (x >= 1) r += 0.5f * (sM1[c - 1] * sP[c - 1]);
        if (x == g.nx - 1) r += 0.5f * (sM1[c] * sP[c]);
        if (x <= g.nx - 2) r -= 0.5f * (sM1[c + 1] * sP[c + 1]);
        if (x == 0) r -= 0.5f * (sM1[c] * sP[c]);
        Ihv += r;
    }
    if (mode == 0) {
        Ih[ob] = Ihv;
        ph[ob] = phv;
    } else {
        const long long ci = ((long long)b * g.ny + y) * g.nx + x;
        if (mode == 1) {
            const float* u0 = slice_of(u, g, 0LL * g.B + b);
            const float* u1 = slice_of(u, g, 1LL * g.B + b);
            float kg = 0.f;
            kg += g0 * u0[o];
            kg += g1 * u1[o];
            const float lam = cf.lambda[b], rho = cf.rho[b];
            out0[ci] = phv + lam * (2.f * kg + 2.f * rho * sP[c]);
        } else {
            out0[ci] = phv;
            if (gI0) gI0[ci] = Ihv;
        }
    }
}

template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_gradp(Geom g, Coefs cf, int t, int mode, const float* __restrict__ states,
            const float* __restrict__ u, const unsigned int* __restrict__ maxdisp,
            const float* __restrict__ mh, float* Ihp, float* php, float* Ih, float* ph,
            float* out0, float* gI0) {
    pdl_wait();  // the previous kernel's writes are visible from here on
    pdl_trigger();
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const int b = v.b;
    const long long o = gidx(g, v.z, v.y, v.x);
    const long long ob = (long long)b * g.inst + o;
    int c[NDIM], n[NDIM];
    long long s[NDIM];
    axis_info<NDIM>(g, v, c, n, s);
    const float* It = slice_of(states, g, ((long long)t * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)t * 2 + 1) * g.B + b);
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
        phv += ma[o] * ga;
        // D_a^T (m^_a p) at this node
        float r = 0.f;
        const long long sa = s[a];
        if (c[a] >= 1) r += 0.5f * (ma[o - sa] * pt[o - sa]);
        if (c[a] == n[a] - 1) r += 0.5f * (ma[o] * pt[o]);
        if (c[a] <= n[a] - 2) r -= 0.5f * (ma[o + sa] * pt[o + sa]);
        if (c[a] == 0) r -= 0.5f * (ma[o] * pt[o]);
        Ihv += r;
        if (mode == 1) kg += ga * slice_of(u, g, (0LL * NDIM + a) * g.B + b)[o];
    }
    if (mode == 0) {
        Ih[ob] = Ihv;
        ph[ob] = phv;
    } else {
        const long long ci = cidx(g, v);
        if (mode == 1) {
            const float lam = cf.lambda[b], rho = cf.rho[b];
            out0[ci] = phv + lam * (2.f * kg + 2.f * rho * pt[o]);
        } else {
            out0[ci] = phv;
            if (gI0) gI0[ci] = Ihv;
        }
    }
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

cudaError_t launch_advect(const Geom& g, int ndim, const Coefs& c, int t, float* states,
                          const float* u, unsigned int* maxdisp, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_advect2d, dim3((g.nx + kPX - 1) / kPX, (g.ny + kPY - 1) / kPY, g.B), blk, 0, st, 
            g, c, t, states, u, maxdisp));
    else
        META_CHECK_LAUNCH(launch_k(k_advect<3>, pgrid<3>(g), blk, 0, st, g, c, t, states, u, maxdisp));
    return cudaGetLastError();
}

cudaError_t launch_cost(const Geom& g, int ndim, const Coefs& c, int T, const float* states,
                        const float* u, const float* J, float* Ih, float* ph, float* Ihp,
                        float* php, double* partials, int nblk, double* cost, cudaStream_t st) {
    const dim3 grid(nblk, g.B);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_cost_partials<2>, grid, 256, 0, st, g, T, states, u, J, Ih, ph, Ihp, php, partials));
    else
        META_CHECK_LAUNCH(launch_k(k_cost_partials<3>, grid, 256, 0, st, g, T, states, u, J, Ih, ph, Ihp, php, partials));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    META_CHECK_LAUNCH(launch_k(k_cost_final, g.B, 256, 0, st, nblk, c, partials, cost));
    return cudaGetLastError();
}

cudaError_t launch_adj_init(const Geom& g, int ndim, const float* gI1, const float* gp1,
                            float* Ih, float* ph, float* Ihp, float* php, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_adj_init<2>, pgrid<2>(g), blk, 0, st, g, gI1, gp1, Ih, ph, Ihp, php));
    else
        META_CHECK_LAUNCH(launch_k(k_adj_init<3>, pgrid<3>(g), blk, 0, st, g, gI1, gp1, Ih, ph, Ihp, php));
    return cudaGetLastError();
}

cudaError_t launch_adj_transport(const Geom& g, int ndim, const Coefs& c, int t,
                                 const float* states, const float* u,
                                 const unsigned int* maxdisp, const float* Ih1, const float* ph1,
                                 float* vh, float* Ihp, float* php, unsigned int* fault,
                                 cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_adj_transport<2>, gather_grid<2>(g), blk, 0, st, g, c, t, states, u, maxdisp, Ih1,
                                                              ph1, vh, Ihp, php, fault));
    else
        META_CHECK_LAUNCH(launch_k(k_adj_transport<3>, gather_grid<3>(g), blk, 0, st, g, c, t, states, u, maxdisp, Ih1,
                                                              ph1, vh, Ihp, php, fault));
    return cudaGetLastError();
}

cudaError_t launch_adj_gradp(const Geom& g, int ndim, const Coefs& c, int t, int mode,
                             const float* states, const float* u, const unsigned int* maxdisp,
                             const float* mh, float* Ihp, float* php, float* Ih, float* ph,
                             float* out0, float* gI0, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        META_CHECK_LAUNCH(launch_k(k_adj_gradp2d, dim3((g.nx + kPX - 1) / kPX, (g.ny + kPY - 1) / kPY, g.B), blk, 0, st, g, c, t, mode, states, u, maxdisp, mh, Ihp,
                                                    php, Ih, ph, out0, gI0));
    else
        META_CHECK_LAUNCH(launch_k(k_adj_gradp<3>, pgrid<3>(g), blk, 0, st, g, c, t, mode, states, u, maxdisp, mh, Ihp,
                                                    php, Ih, ph, out0, gI0));
    return cudaGetLastError();
}

}  // namespace meta
