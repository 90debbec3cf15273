// meta_step.cu -- pointwise and gather kernels of the semi-Lagrangian step and
// of its discrete adjoint (arXiv:2106.08817, Eq. 3-4, Sec. 2.3), sm_103a.
//
// Forward step t (after the blur passes have produced u_t = K(p_t grad I_t)):
//   k_advect      div v, foot y = x - dt v (v = -rho u), bi/trilinear gathers of
//                 I_t and p_t, p_{t+1} = p~ (1 - dt div v), I_{t+1} = I~ + dt mu p~,
//                 and the per-instance max displacement (window of the adjoint).
// Adjoint step t (reverse), the transpose of the step above:
//   k_adj_pre     per source x: p~^ = p^'(1 - dt div v) + dt mu I^', div^ = -dt p~ p^'
//   k_adj_gather  per node n: S^T by gather over the sources whose foot cell
//                 touches n (fixed order, no atomics), the foot derivative y^,
//                 and v^ = -dt y^ + D^T div^
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

// (D^T w)[c] along a stride s: rows c-1 and c+1 of D, plus the edge rows.
__device__ __forceinline__ float cdiff_T(const float* w, long long o, long long s, int c, int n) {
    float r = 0.f;
    if (c >= 1) r += 0.5f * w[o - s];
    if (c == n - 1) r += 0.5f * w[o];
    if (c <= n - 2) r -= 0.5f * w[o + s];
    if (c == 0) r -= 0.5f * w[o];
    return r;
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
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
    const long long o = (long long)v.b * g.inst + gidx(g, v.z, v.y, v.x);
    const long long ci = cidx(g, v);
    if (I1) I1[ci] = sI[o];
    if (p1) p1[ci] = sP[o];
}

template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_advect(Geom g, Coefs cf, int t, float* __restrict__ states, const float* __restrict__ u,
         unsigned int* __restrict__ maxdisp) {
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
    // per-instance max |displacement| (non-negative floats order like their bits)
    const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(dmax));
    if ((threadIdx.x & 31) == 0 && m != 0u)
        atomicMax(maxdisp + (long long)t * g.B + blockIdx.z, m);
}

// Cost partials: one CTA = 256 threads over a fixed voxel range of instance
// blockIdx.y; also writes the adjoint start I^_T = I_T - J, p^_T = 0.
template <int NDIM>
__global__ void __launch_bounds__(256)
k_cost_partials(Geom g, int T, const float* __restrict__ states, const float* __restrict__ u,
                const float* __restrict__ J, float* Ih, float* ph, float* Ihp, float* php,
                double* partials) {
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
    return 1 + (int)floorf(__uint_as_float(maxdisp[(long long)t * B + b]));
}

template <int NDIM>
struct GatherTile;  // node tile of the gather kernel (256 nodes per CTA)
template <>
struct GatherTile<2> {
    static constexpr int TX = 32, TY = 8, TZ = 1, RMAX = 8;
};
template <>
struct GatherTile<3> {
    static constexpr int TX = 8, TY = 8, TZ = 4, RMAX = 3;
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

template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_pre(Geom g, Coefs cf, int t, const float* __restrict__ states, const float* __restrict__ u,
          const unsigned int* __restrict__ maxdisp, const float* __restrict__ Ih1,
          const float* __restrict__ ph1, float* pth, float* dh, float* Ihp, float* php,
          unsigned int* fault) {
    const Vox v = vox_of<NDIM>(g);
    if (!v.ok) return;
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
    }
    const float div = -rho * du;
    const Feet<NDIM> F = feet_of<NDIM>(g, v, d);
    const float* pt = slice_of(states, g, ((long long)t * 2 + 1) * g.B + b);
    const float pw = interp<NDIM>(g, F, pt);
    const long long ob = (long long)b * g.inst + o;
    const float phv = ph1[ob];
    const float Ihv = Ih1[ob];
    const float pthv = phv * (1.f - dt * div) + (dt * mu) * Ihv;
    pth[ob] = pthv;
    dh[ob] = -dt * pw * phv;
    if (gather_radius(maxdisp, t, g.B, b) > GatherTile<NDIM>::RMAX) {
        // Displacements beyond the gather window: scatter S^T with atomics
        // (work bounded by 2^d per source; summation order not fixed).
        if (o == 0) atomicOr(fault, kInfoScatter);
        float* Ib = Ihp + (long long)b * g.inst;
        float* Pb = php + (long long)b * g.inst;
#pragma unroll
        for (int k = 0; k < (1 << NDIM); ++k) {
            float w = 1.f;
            long long q = F.base;
#pragma unroll
            for (int a = 0; a < NDIM; ++a) {
                const int up = (k >> a) & 1;
                w *= up ? F.f[a].f : 1.f - F.f[a].f;
                q += up ? s[a] : 0;
            }
            atomicAdd(Ib + q, w * Ihv);
            atomicAdd(Pb + q, w * pthv);
        }
    }
}

// Packs the foot cell of a source relative to the source (one byte per axis,
// offset + 64) with bit 31 set for sources outside the domain.
__device__ __forceinline__ int pack_cell(const int* off) {
    return (off[0] + 64) | ((off[1] + 64) << 8) | ((off[2] + 64) << 16);
}

template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_gather(Geom g, Coefs cf, int t, const float* __restrict__ states,
             const float* __restrict__ u, const unsigned int* __restrict__ maxdisp,
             const float* __restrict__ Ih1, const float* __restrict__ pth,
             const float* __restrict__ dh, float* vh, float* Ihp, float* php) {
    using G = GatherTile<NDIM>;
    constexpr int REG = gather_region<NDIM>();
    __shared__ int s_cell[REG];
    __shared__ float s_f[NDIM][REG];
    __shared__ float s_I[REG];
    __shared__ float s_P[REG];

    const int b = blockIdx.z;
    const float rho = cf.rho[b], dt = cf.dt;
    const float dtrho = dt * rho;
    const int tid = threadIdx.y * kPX + threadIdx.x;
    const int ntx = (g.ny + G::TY - 1) / G::TY;
    const int x0 = blockIdx.x * G::TX;
    const int y0 = (blockIdx.y % ntx) * G::TY;
    const int z0 = (blockIdx.y / ntx) * G::TZ;
    // this thread's node
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
    const float* ub[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) ub[a] = slice_of(u, g, ((long long)t * NDIM + a) * g.B + b);
    const float* Ihb = Ih1 + (long long)b * g.inst;
    const float* pthb = pth + (long long)b * g.inst;
    const float* dhb = dh + (long long)b * g.inst;
    const int R = gather_radius(maxdisp, t, g.B, b);
    const bool tiled = R <= G::RMAX;  // uniform over the CTA

    float accI = 0.f, accP = 0.f;
    if (tiled) {
        // Phase 1: foot records of every source of the tile grown by R.
        const int RX = G::TX + 2 * R, RY = G::TY + 2 * R;
        const int RZ = (NDIM == 3) ? G::TZ + 2 * R : 1;
        const int nreg = RX * RY * RZ;
        for (int i = tid; i < nreg; i += kPX * kPY) {
            const int rx = i % RX;
            const int ry = (i / RX) % RY;
            const int rz = i / (RX * RY);
            const int sx = x0 - R + rx, sy = y0 - R + ry;
            const int sz = (NDIM == 3) ? z0 - R + rz : 0;
            int cell = (int)0x80000000;
            float fI = 0.f, fP = 0.f;
            float ff[NDIM];
#pragma unroll
            for (int a = 0; a < NDIM; ++a) ff[a] = 0.f;
            if (sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz) {
                const long long so = gidx(g, sz, sy, sx);
                int off[3] = {0, 0, 0};
                if constexpr (NDIM == 2) {
                    const Foot1 fy = foot1(sy, disp_of(dtrho, ub[0][so]), g.ny);
                    const Foot1 fx = foot1(sx, disp_of(dtrho, ub[1][so]), g.nx);
                    off[0] = fy.i0 - sy;
                    off[1] = fx.i0 - sx;
                    ff[0] = fy.f;
                    ff[1] = fx.f;
                } else {
                    const Foot1 fz = foot1(sz, disp_of(dtrho, ub[0][so]), g.nz);
                    const Foot1 fy = foot1(sy, disp_of(dtrho, ub[1][so]), g.ny);
                    const Foot1 fx = foot1(sx, disp_of(dtrho, ub[2][so]), g.nx);
                    off[0] = fz.i0 - sz;
                    off[1] = fy.i0 - sy;
                    off[2] = fx.i0 - sx;
                    ff[0] = fz.f;
                    ff[1] = fy.f;
                    ff[2] = fx.f;
                }
                cell = pack_cell(off);
                fI = Ihb[so];
                fP = pthb[so];
            }
            s_cell[i] = cell;
#pragma unroll
            for (int a = 0; a < NDIM; ++a) s_f[a][i] = ff[a];
            s_I[i] = fI;
            s_P[i] = fP;
        }
        __syncthreads();
        // Phase 2: S^T by gather over the window, fixed order, no atomics.
        if (v.ok) {
            const int lx = v.x - x0 + R, ly = v.y - y0 + R;
            const int lz = (NDIM == 3) ? v.z - z0 + R : 0;
            for (int dz = (NDIM == 3 ? -R : 0); dz <= (NDIM == 3 ? R : 0); ++dz) {
                for (int dy = -R; dy <= R; ++dy) {
                    const int rowbase = ((lz + dz) * RY + (ly + dy)) * RX + lx;
                    for (int dx = -R; dx <= R; ++dx) {
                        const int i = rowbase + dx;
                        const int cell = s_cell[i];
                        // node - source - offset must be 0 or 1 on every axis
                        const int ex = -dx - (((cell >> ((NDIM - 1) * 8)) & 0xff) - 64);
                        const int ey = -dy - (((cell >> ((NDIM - 2) * 8)) & 0xff) - 64);
                        int ez = 0;
                        if constexpr (NDIM == 3) ez = -dz - ((cell & 0xff) - 64);
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
                        accI += w * s_I[i];
                        accP += w * s_P[i];
                    }
                }
            }
        }
    }
    if (!v.ok) return;
    const long long o = gidx(g, v.z, v.y, v.x);
    const long long ob = (long long)b * g.inst + o;
    if (tiled) {
        Ihp[ob] = accI;
        php[ob] = accP;
    }  // else: k_adj_pre scattered S^T into Ihp / php already

    int c[NDIM], n[NDIM];
    long long s[NDIM];
    axis_info<NDIM>(g, v, c, n, s);
    // Foot derivative of this node's own backtracking: y^_a.
    float d[NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) d[a] = disp_of(dtrho, ub[a][o]);
    const Feet<NDIM> F = feet_of<NDIM>(g, v, d);
    const float* It = slice_of(states, g, ((long long)t * 2 + 0) * g.B + b);
    const float* pt = slice_of(states, g, ((long long)t * 2 + 1) * g.B + b);
    float Iv, pv, dI[NDIM], dP[NDIM];
    interp_grad<NDIM>(g, F, It, &Iv, dI);
    interp_grad<NDIM>(g, F, pt, &pv, dP);
    const float Ihv = Ihb[o], pthv = pthb[o];
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const float yh = dI[a] * Ihv + dP[a] * pthv;
        const float vha = -dt * yh + cdiff_T(dhb, o, s[a], c[a], n[a]);
        vh[((long long)a * g.B + b) * g.inst + o] = vha;
    }
}

template <int NDIM>
__global__ void __launch_bounds__(kPX * kPY)
k_adj_gradp(Geom g, Coefs cf, int t, int mode, const float* __restrict__ states,
            const float* __restrict__ u, const unsigned int* __restrict__ maxdisp,
            const float* __restrict__ mh, float* Ihp, float* php, float* Ih, float* ph,
            float* out0, float* gI0) {
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
        k_pack<2><<<pgrid<2>(g), blk, 0, st>>>(g, I0, p0, dI, dP);
    else
        k_pack<3><<<pgrid<3>(g), blk, 0, st>>>(g, I0, p0, dI, dP);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Geom& g, int ndim, const float* sI, const float* sP, float* I1,
                          float* p1, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        k_unpack<2><<<pgrid<2>(g), blk, 0, st>>>(g, sI, sP, I1, p1);
    else
        k_unpack<3><<<pgrid<3>(g), blk, 0, st>>>(g, sI, sP, I1, p1);
    return cudaGetLastError();
}

cudaError_t launch_advect(const Geom& g, int ndim, const Coefs& c, int t, float* states,
                          const float* u, unsigned int* maxdisp, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        k_advect<2><<<pgrid<2>(g), blk, 0, st>>>(g, c, t, states, u, maxdisp);
    else
        k_advect<3><<<pgrid<3>(g), blk, 0, st>>>(g, c, t, states, u, maxdisp);
    return cudaGetLastError();
}

cudaError_t launch_cost(const Geom& g, int ndim, const Coefs& c, int T, const float* states,
                        const float* u, const float* J, float* Ih, float* ph, float* Ihp,
                        float* php, double* partials, int nblk, double* cost, cudaStream_t st) {
    const dim3 grid(nblk, g.B);
    if (ndim == 2)
        k_cost_partials<2><<<grid, 256, 0, st>>>(g, T, states, u, J, Ih, ph, Ihp, php, partials);
    else
        k_cost_partials<3><<<grid, 256, 0, st>>>(g, T, states, u, J, Ih, ph, Ihp, php, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_cost_final<<<g.B, 256, 0, st>>>(nblk, c, partials, cost);
    return cudaGetLastError();
}

cudaError_t launch_adj_init(const Geom& g, int ndim, const float* gI1, const float* gp1,
                            float* Ih, float* ph, float* Ihp, float* php, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        k_adj_init<2><<<pgrid<2>(g), blk, 0, st>>>(g, gI1, gp1, Ih, ph, Ihp, php);
    else
        k_adj_init<3><<<pgrid<3>(g), blk, 0, st>>>(g, gI1, gp1, Ih, ph, Ihp, php);
    return cudaGetLastError();
}

cudaError_t launch_adj_pre(const Geom& g, int ndim, const Coefs& c, int t, const float* states,
                           const float* u, const unsigned int* maxdisp, const float* Ih1,
                           const float* ph1, float* pth, float* dh, float* Ihp, float* php,
                           unsigned int* fault, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        k_adj_pre<2><<<pgrid<2>(g), blk, 0, st>>>(g, c, t, states, u, maxdisp, Ih1, ph1, pth, dh,
                                                  Ihp, php, fault);
    else
        k_adj_pre<3><<<pgrid<3>(g), blk, 0, st>>>(g, c, t, states, u, maxdisp, Ih1, ph1, pth, dh,
                                                  Ihp, php, fault);
    return cudaGetLastError();
}

cudaError_t launch_adj_gather(const Geom& g, int ndim, const Coefs& c, int t,
                              const float* states, const float* u, const unsigned int* maxdisp,
                              const float* Ih1, const float* pth, const float* dh, float* vh,
                              float* Ihp, float* php, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        k_adj_gather<2><<<gather_grid<2>(g), blk, 0, st>>>(g, c, t, states, u, maxdisp, Ih1, pth,
                                                           dh, vh, Ihp, php);
    else
        k_adj_gather<3><<<gather_grid<3>(g), blk, 0, st>>>(g, c, t, states, u, maxdisp, Ih1, pth,
                                                           dh, vh, Ihp, php);
    return cudaGetLastError();
}

cudaError_t launch_adj_gradp(const Geom& g, int ndim, const Coefs& c, int t, int mode,
                             const float* states, const float* u, const unsigned int* maxdisp,
                             const float* mh, float* Ihp, float* php, float* Ih, float* ph,
                             float* out0, float* gI0, cudaStream_t st) {
    const dim3 blk(kPX, kPY);
    if (ndim == 2)
        k_adj_gradp<2><<<pgrid<2>(g), blk, 0, st>>>(g, c, t, mode, states, u, maxdisp, mh, Ihp,
                                                    php, Ih, ph, out0, gI0);
    else
        k_adj_gradp<3><<<pgrid<3>(g), blk, 0, st>>>(g, c, t, mode, states, u, maxdisp, mh, Ihp,
                                                    php, Ih, ph, out0, gI0);
    return cudaGetLastError();
}

}  // namespace meta
