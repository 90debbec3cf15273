// meta_stencil.cuh -- device helpers shared by the forward and adjoint kernels
// of the semi-Lagrangian step: voxel indexing, central differences, the
// displacement of a foot, cp.async staging, bi/trilinear interpolation and
// its derivatives.
#pragma once

#include "meta_kernels.h"

namespace meta {
namespace {

constexpr int kPX = 32, kPY = 8;  // pointwise block

struct Vox {
    int b, z, y, x;
    bool ok;
};

template <int NDIM, class K>
__device__ __forceinline__ Vox vox_of(const Geom& g, const K& kb) {
    Vox v;
    const int nyt = (g.ny + kPY - 1) / kPY;
    const int zq = (NDIM == 3) ? div_nyt(g, kb.by()) : 0;
    v.b = kb.bz();
    v.x = kb.bx() * kPX + kb.tx();
    v.y = (kb.by() - zq * nyt) * kPY + kb.ty();
    v.z = zq;
    v.ok = v.x < g.nx && v.y < g.ny && v.z < g.nz;
    return v;
}
template <int NDIM>
__device__ __forceinline__ Vox vox_of(const Geom& g) {
    return vox_of<NDIM>(g, HwBlk{});
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
                                            const Geom& g, int xlo, int ylo, int tid) {
    constexpr int NC4 = W / 4;
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

// Record arithmetic of the adjoint with every rounding explicit (no FMA
// contraction), so that every kernel that builds a record of a step -- from
// staged tiles or from global memory -- writes the same bits.
__device__ __forceinline__ float rn_cdiff(float hi, float lo) {
    return __fmul_rn(0.5f, __fsub_rn(hi, lo));
}
__device__ __forceinline__ float rn_lerp(float a, float b, float f) {
    return __fadd_rn(__fmul_rn(__fsub_rn(1.f, f), a), __fmul_rn(f, b));
}
__device__ __forceinline__ float rn_bilin(const float* p, long long W, float fy, float fx) {
    return rn_lerp(rn_lerp(p[0], p[1], fx), rn_lerp(p[W], p[W + 1], fx), fy);
}
__device__ __forceinline__ float rn_trilin(const float* p, const float* q, long long P, float fz,
                                           float fy, float fx) {
    const float b0 = rn_lerp(rn_lerp(p[0], p[1], fx), rn_lerp(p[P], p[P + 1], fx), fy);
    const float b1 = rn_lerp(rn_lerp(q[0], q[1], fx), rn_lerp(q[P], q[P + 1], fx), fy);
    return rn_lerp(b0, b1, fz);
}
// p~^ = p^' (1 - dt div) + dt mu I^'  and  div^ = -dt p~ p^'
__device__ __forceinline__ float rn_ptilde_hat(float ph1, float Ih1, float dt, float mu,
                                               float div) {
    return __fadd_rn(__fmul_rn(ph1, __fsub_rn(1.f, __fmul_rn(dt, div))),
                     __fmul_rn(__fmul_rn(dt, mu), Ih1));
}
__device__ __forceinline__ float rn_div_hat(float dt, float pw, float ph1) {
    return __fmul_rn(__fmul_rn(-dt, pw), ph1);
}

// Exact Jacobian of the backtrack Id - dt v with v = -rho u:
// J = det(Id + dt rho A), A[a][e] = D_e u_a, every rounding explicit so that
// the forward step and every record builder compute the same bits.
template <int NDIM>
__device__ __forceinline__ float rn_jac_det(const float (&A)[NDIM][NDIM], float dtrho) {
    float M[NDIM][NDIM];
#pragma unroll
    for (int a = 0; a < NDIM; ++a)
#pragma unroll
        for (int e = 0; e < NDIM; ++e)
            M[a][e] = __fadd_rn(a == e ? 1.f : 0.f, __fmul_rn(dtrho, A[a][e]));
    if constexpr (NDIM == 2) {
        return __fsub_rn(__fmul_rn(M[0][0], M[1][1]), __fmul_rn(M[0][1], M[1][0]));
    } else {
        const float c0 = __fsub_rn(__fmul_rn(M[1][1], M[2][2]), __fmul_rn(M[1][2], M[2][1]));
        const float c1 = __fsub_rn(__fmul_rn(M[1][0], M[2][2]), __fmul_rn(M[1][2], M[2][0]));
        const float c2 = __fsub_rn(__fmul_rn(M[1][0], M[2][1]), __fmul_rn(M[1][1], M[2][0]));
        return __fadd_rn(__fsub_rn(__fmul_rn(M[0][0], c0), __fmul_rn(M[0][1], c1)),
                         __fmul_rn(M[0][2], c2));
    }
}
// p~^ = p^' J + dt mu I^'  (the det update)
__device__ __forceinline__ float rn_ptilde_hat_J(float ph1, float Ih1, float dt, float mu,
                                                 float J) {
    return __fadd_rn(__fmul_rn(ph1, J), __fmul_rn(__fmul_rn(dt, mu), Ih1));
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
        F.f[0] = foot1g(g, v.y, d[0], g.ny);
        F.f[1] = foot1g(g, v.x, d[1], g.nx);
        F.base = gidx(g, 0, F.f[0].i0, F.f[1].i0);
    } else {
        F.f[0] = foot1g(g, v.z, d[0], g.nz);
        F.f[1] = foot1g(g, v.y, d[1], g.ny);
        F.f[2] = foot1g(g, v.x, d[2], g.nx);
        F.base = gidx(g, F.f[0].i0, F.f[1].i0, F.f[2].i0);
    }
    return F;
}

// Trilinear value at lower corner p[0] with row stride P and plane stride S
// (global or shared memory); the same expressions everywhere.
template <typename I>
__device__ __forceinline__ float trilin(const float* p, I P, I S, float fz, float fy, float fx) {
    const float a0 = (1.f - fx) * p[0] + fx * p[1];
    const float a1 = (1.f - fx) * p[P] + fx * p[P + 1];
    const float a2 = (1.f - fx) * p[S] + fx * p[S + 1];
    const float a3 = (1.f - fx) * p[S + P] + fx * p[S + P + 1];
    const float b0 = (1.f - fy) * a0 + fy * a1;
    const float b1 = (1.f - fy) * a2 + fy * a3;
    return (1.f - fz) * b0 + fz * b1;
}

// Trilinear value with the lower z plane at p and the upper at q (the same
// expressions as trilin).
template <typename I>
__device__ __forceinline__ float trilin_pq(const float* p, const float* q, I P, float fz,
                                           float fy, float fx) {
    const float a0 = (1.f - fx) * p[0] + fx * p[1];
    const float a1 = (1.f - fx) * p[P] + fx * p[P + 1];
    const float a2 = (1.f - fx) * q[0] + fx * q[1];
    const float a3 = (1.f - fx) * q[P] + fx * q[P + 1];
    const float b0 = (1.f - fy) * a0 + fy * a1;
    const float b1 = (1.f - fy) * a2 + fy * a3;
    return (1.f - fz) * b0 + fz * b1;
}

// Trilinear value and its derivatives along z, y, x (zero where the clamp on
// that axis is active), with the lower z plane at p and the upper at q.
template <typename I>
__device__ __forceinline__ void trilin_grad_pq(const float* p, const float* q, I P, float fz,
                                               float fy, float fx, bool inz, bool iny, bool inx,
                                               float* val, float* dv) {
    const float c000 = p[0], c001 = p[1], c010 = p[P], c011 = p[P + 1];
    const float c100 = q[0], c101 = q[1], c110 = q[P], c111 = q[P + 1];
    const float a0 = (1.f - fx) * c000 + fx * c001;
    const float a1 = (1.f - fx) * c010 + fx * c011;
    const float a2 = (1.f - fx) * c100 + fx * c101;
    const float a3 = (1.f - fx) * c110 + fx * c111;
    const float b0 = (1.f - fy) * a0 + fy * a1;
    const float b1 = (1.f - fy) * a2 + fy * a3;
    *val = (1.f - fz) * b0 + fz * b1;
    dv[0] = inz ? (b1 - b0) : 0.f;
    dv[1] = iny ? ((1.f - fz) * (a1 - a0) + fz * (a3 - a2)) : 0.f;
    const float e0 = (1.f - fy) * (c001 - c000) + fy * (c011 - c010);
    const float e1 = (1.f - fy) * (c101 - c100) + fy * (c111 - c110);
    dv[2] = inx ? ((1.f - fz) * e0 + fz * e1) : 0.f;
}
template <typename I>
__device__ __forceinline__ void trilin_grad(const float* p, I P, I S, float fz, float fy,
                                            float fx, bool inz, bool iny, bool inx, float* val,
                                            float* dv) {
    trilin_grad_pq<I>(p, p + S, P, fz, fy, fx, inz, iny, inx, val, dv);
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
        return trilin<long long>(p, g.P, g.slab, F.f[0].f, F.f[1].f, F.f[2].f);
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
        trilin_grad<long long>(p, g.P, g.slab, F.f[0].f, F.f[1].f, F.f[2].f, F.f[0].inside,
                               F.f[1].inside, F.f[2].inside, val, dv);
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

}  // namespace
}  // namespace meta
