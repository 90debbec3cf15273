// meta_lbfgs.cu -- L-BFGS over the cost of Eq. 4 (the quasi-Newton option the
// paper mentions beside gradient descent, Sec. 3), sm_103a.
//
// The inverse-Hessian product is the two-loop recursion (Nocedal & Wright,
// Numerical Optimization, Algorithm 7.4) over the last m pairs
// s_i = x_{i+1} - x_i, y_i = g_{i+1} - g_i of each instance, with
// H_0 = gamma I, gamma = s^T y / y^T y of the newest usable pair.  Every vector
// operation runs on the device: FP64 dot products with a fixed summation order
// (per-CTA partials over fixed chunks, then one CTA per instance), FP32 axpys
// whose coefficients stay on the device, so a direction needs no host round
// trip.  meta_lbfgs_minimize keeps every per-instance decision on the device
// too (the choice of direction, the Armijo test and halving of the
// backtracking line search, stopping, the new pair's rho and gamma); the host
// loop only launches, and reads one small block per line-search trial (how
// many instances still search, and the costs): one read per iteration when
// the first step is accepted.
#include <climits>
#include <cstddef>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "meta.h"
#include "meta_common.cuh"

namespace meta {
namespace {

constexpr int kLT = 256;       // threads per CTA
constexpr long long kStateMagic = 0x53464c4241544d45LL;  // marks a valid state header
constexpr int kLMaxBlk = 512;  // dot-product CTAs per instance

int dot_blocks(long long N) {
    long long nb = (N + kLT * 8 - 1) / (kLT * 8);
    if (nb < 1) nb = 1;
    if (nb > kLMaxBlk) nb = kLMaxBlk;
    return (int)nb;
}

// Per-CTA FP64 partial sums of a[b] . b[b] (or of max |a[b]| when MAX) over a
// fixed chunk of instance b; partials[b * nb + blk].
template <bool MAX>
__global__ void __launch_bounds__(kLT)
k_ldot(long long N, const float* __restrict__ a, const float* __restrict__ b, double* partials) {
    const int inst = blockIdx.y, nb = gridDim.x;
    const long long chunk = (N + nb - 1) / nb;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < N ? lo + chunk : N;
    const float* pa = a + (long long)inst * N;
    const float* pb = b ? b + (long long)inst * N : nullptr;
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kLT) {
        if constexpr (MAX) acc = fmax(acc, (double)fabsf(pa[i]));
        else acc += (double)pa[i] * (double)pb[i];
    }
    __shared__ double red[kLT];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kLT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            red[threadIdx.x] = MAX ? fmax(red[threadIdx.x], red[threadIdx.x + w])
                                   : red[threadIdx.x] + red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[(long long)inst * nb + blockIdx.x] = red[0];
}

// out[b] = the partials of instance b combined in a fixed order.
template <bool MAX>
__global__ void __launch_bounds__(kLT)
k_lred(int nb, const double* __restrict__ partials, double* out) {
    const int inst = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kLT) {
        const double v = partials[(long long)inst * nb + i];
        acc = MAX ? fmax(acc, v) : acc + v;
    }
    __shared__ double red[kLT];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kLT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            red[threadIdx.x] = MAX ? fmax(red[threadIdx.x], red[threadIdx.x + w])
                                   : red[threadIdx.x] + red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[inst] = red[0];
}

// Coefficients of the two-loop recursion, one thread per instance:
//   mode 0 (first loop):  alpha_i = rho_i (s_i . q),   coef = -alpha_i
//   mode 1 (second loop): beta = rho_i (y_i . r),      coef = alpha_i - beta
__global__ void k_lcoef(int B, int mode, const double* __restrict__ rho_i, double* alpha_i,
                        const double* __restrict__ dot, double* coef) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (mode == 0) {
        alpha_i[b] = rho_i[b] * dot[b];
        coef[b] = -alpha_i[b];
    } else {
        coef[b] = alpha_i[b] - rho_i[b] * dot[b];
    }
}

// y[b] += coef[b] x[b]  (coef rounded to FP32 once per instance)
__global__ void __launch_bounds__(kLT)
k_laxpy(long long N, const double* __restrict__ coef, const float* __restrict__ x, float* y) {
    const int b = blockIdx.y;
    const float c = (float)coef[b];
    const long long o = (long long)b * N;
    for (long long i = (long long)blockIdx.x * kLT + threadIdx.x; i < N;
         i += (long long)gridDim.x * kLT)
        y[o + i] = fmaf(c, x[o + i], y[o + i]);
}

// y[b] *= coef[b]
__global__ void __launch_bounds__(kLT)
k_lscale(long long N, const double* __restrict__ coef, float* y) {
    const int b = blockIdx.y;
    const float c = (float)coef[b];
    const long long o = (long long)b * N;
    for (long long i = (long long)blockIdx.x * kLT + threadIdx.x; i < N;
         i += (long long)gridDim.x * kLT)
        y[o + i] *= c;
}

// d[b] = c[b] g[b] where use[b] (a scaled steepest-descent step)
__global__ void __launch_bounds__(kLT)
k_lsteep(long long N, const int* __restrict__ use, const double* __restrict__ c,
         const float* __restrict__ g, float* d) {
    const int b = blockIdx.y;
    if (!use[b]) return;
    const float cb = (float)c[b];
    const long long o = (long long)b * N;
    for (long long i = (long long)blockIdx.x * kLT + threadIdx.x; i < N;
         i += (long long)gridDim.x * kLT)
        d[o + i] = cb * g[o + i];
}

// where keep[b]: xa[b] = xt[b], ga[b] = gt[b] (the accepted trial point)
__global__ void __launch_bounds__(kLT)
k_lkeep(long long N, const int* __restrict__ keep, const float* __restrict__ xt,
        const float* __restrict__ gt, float* xa, float* ga) {
    const int b = blockIdx.y;
    if (!keep[b]) return;
    const long long o = (long long)b * N;
    for (long long i = (long long)blockIdx.x * kLT + threadIdx.x; i < N;
         i += (long long)gridDim.x * kLT) {
        xa[o + i] = xt[o + i];
        ga[o + i] = gt[o + i];
    }
}

// New pair: where moved[b], s = xa - x, y = ga - g, then x = xa, g = ga;
// elsewhere s = y = 0 (a pair with rho = 0 has no effect).
__global__ void __launch_bounds__(kLT)
k_lpair(long long N, const int* __restrict__ moved, float* x, float* g,
        const float* __restrict__ xa, const float* __restrict__ ga, float* s, float* y) {
    const int b = blockIdx.y;
    const bool mv = moved[b] != 0;
    const long long o = (long long)b * N;
    for (long long i = (long long)blockIdx.x * kLT + threadIdx.x; i < N;
         i += (long long)gridDim.x * kLT) {
        if (mv) {
            s[o + i] = xa[o + i] - x[o + i];
            y[o + i] = ga[o + i] - g[o + i];
            x[o + i] = xa[o + i];
            g[o + i] = ga[o + i];
        } else {
            s[o + i] = 0.f;
            y[o + i] = 0.f;
        }
    }
}

// d[b] = -d[b]
__global__ void __launch_bounds__(kLT)
k_lneg(long long N, int B, float* d) {
    const int b = blockIdx.y;
    const long long o = (long long)b * N;
    for (long long i = (long long)blockIdx.x * kLT + threadIdx.x; i < N;
         i += (long long)gridDim.x * kLT)
        d[o + i] = -d[o + i];
}

// Per-instance state of meta_lbfgs_minimize, all on the device (one thread
// per instance in the kernels below).
struct LSt {
    double *L, *gd, *gmax, *gg, *step, *coef, *sy, *yy, *rho, *gamma, *cost;
    int *use, *keep, *accepted, *stopped, *searching, *done;
    unsigned long long* any;  // an instance is still searching (read by the host)
};

// After the first cost_and_grad: L = the sum of the three terms of Eq. 4.
__global__ void k_linit(int B, LSt st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    st.L[b] = st.cost[3 * b] + st.cost[3 * b + 1] + st.cost[3 * b + 2];
    st.stopped[b] = 0;
    st.done[b] = 0;
    st.gamma[b] = 1.0;
}

// The direction of iteration k, from gd = g.d, gmax = max |g|, gg = g.g: an
// instance without a usable pair, or whose d does not descend, takes the scaled
// steepest-descent step -h0 g / max|g| and forgets its pairs; the line search
// starts at step 1 (step 0 and stop where there is no descent).
__global__ void k_ldecide(int B, int m, float h0, LSt st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    int nvalid = 0;
    for (int i = 0; i < m; ++i) nvalid += st.rho[(size_t)i * B + b] != 0.0;
    const int use = (!st.stopped[b] && (nvalid == 0 || !(st.gd[b] < 0.0))) ? 1 : 0;
    st.use[b] = use;
    st.coef[b] = st.gmax[b] > 0.0 ? -(double)h0 / st.gmax[b] : 0.0;
    if (use) {
        st.gd[b] = st.coef[b] * st.gg[b];
        for (int i = 0; i < m; ++i) st.rho[(size_t)i * B + b] = 0.0;  // forget
        st.gamma[b] = 1.0;
    }
    st.accepted[b] = 0;
    st.step[b] = (st.stopped[b] || !(st.gd[b] < 0.0)) ? 0.0 : 1.0;
    if (st.step[b] == 0.0) st.stopped[b] = 1;
    st.searching[b] = !st.stopped[b];
}

// xt[b] = x[b] + step[b] d[b] where the instance is still searching, else x[b]
__global__ void __launch_bounds__(kLT)
k_ltrial2(long long N, LSt st, const float* __restrict__ x, const float* __restrict__ d,
          float* xt) {
    const int b = blockIdx.y;
    const float a = st.searching[b] ? (float)st.step[b] : 0.f;
    const long long o = (long long)b * N;
    for (long long i = (long long)blockIdx.x * kLT + threadIdx.x; i < N;
         i += (long long)gridDim.x * kLT)
        xt[o + i] = a == 0.f ? x[o + i] : fmaf(a, d[o + i], x[o + i]);
}

// Armijo test of the trial (its costs in st.cost): accept the first step with
// L(x + a d) <= L(x) + c1 a g.d, else halve it; `any` counts the instances
// still searching (cleared before).
__global__ void k_larmijo(int B, double c1, LSt st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    st.keep[b] = 0;
    if (st.searching[b]) {
        const double Lt = st.cost[3 * b] + st.cost[3 * b + 1] + st.cost[3 * b + 2];
        if (Lt <= st.L[b] + c1 * st.step[b] * st.gd[b]) {
            st.accepted[b] = 1;
            st.keep[b] = 1;
            st.L[b] = Lt;
            st.searching[b] = 0;
        } else {
            st.step[b] *= 0.5;
        }
    }
    if (st.searching[b]) atomicAdd(st.any, 1ull);
}

// End of iteration k: an instance whose search found no decrease keeps its
// iterate and stops.
__global__ void k_lfinish(int B, LSt st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (!st.accepted[b]) st.stopped[b] = 1;
}

// The new pair's rho = 1 / s.y (0 when s.y <= 1e-12 y.y: unused) and gamma.
__global__ void k_lrho(int B, int head, int k, LSt st) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const bool acc = st.accepted[b] != 0;
    const bool ok = acc && st.sy[b] > 1e-12 * st.yy[b] && st.yy[b] > 0.0;
    st.rho[(size_t)head * B + b] = ok ? 1.0 / st.sy[b] : 0.0;
    if (ok) st.gamma[b] = st.sy[b] / st.yy[b];
    if (acc) st.done[b] = k + 1;
}

// Gradient-descent step size per instance: coef = -h0 / max|g| (0 where g = 0).
__global__ void k_lgdcoef(int B, float h0, const double* __restrict__ gmax, double* coef) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    coef[b] = gmax[b] > 0.0 ? -(double)h0 / gmax[b] : 0.0;
}

dim3 vec_grid(long long N, int B) {
    long long gx = (N + kLT * 4 - 1) / (kLT * 4);
    if (gx < 1) gx = 1;
    if (gx > 4096) gx = 4096;
    return dim3((unsigned)gx, (unsigned)B);
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// L-BFGS workspace map for B instances of N voxels and m pairs.
struct LMap {
    long long N;
    int B, m, nb;
    size_t oS, oY, oG, oGt, oXt, oXa, oGa, oD;        // float vectors
    size_t oRho, oAlpha, oGamma, oDot, oCoef, oStep, oPart, oCost;  // doubles
    size_t oRead;                                   // {searching count, L[B]}: the host's read
    size_t oGd, oGmax, oGg, oSy, oYy;               // doubles [B]
    size_t oUse, oKeep, oAcc, oStop, oSearch, oDone;  // ints [B]
    size_t oHdr;  // long long [4]: {kStateMagic, iterations done, pairs held, ring head}
    size_t total;
};

LMap lbfgs_map(long long N, int B, int m) {
    LMap M;
    std::memset(&M, 0, sizeof(M));
    M.N = N;
    M.B = B;
    M.m = m;
    M.nb = dot_blocks(N);
    const size_t vec = up256(sizeof(float) * (size_t)N * B);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += up256(bytes);
        return o;
    };
    M.oS = take(vec * m);
    M.oY = take(vec * m);
    M.oG = take(vec);
    M.oGt = take(vec);
    M.oXt = take(vec);
    M.oXa = take(vec);
    M.oGa = take(vec);
    M.oD = take(vec);
    M.oRho = take(sizeof(double) * (size_t)m * B);
    M.oAlpha = take(sizeof(double) * (size_t)m * B);
    M.oGamma = take(sizeof(double) * B);
    M.oDot = take(sizeof(double) * B);
    M.oCoef = take(sizeof(double) * B);
    M.oStep = take(sizeof(double) * B);
    M.oPart = take(sizeof(double) * (size_t)B * M.nb);
    M.oCost = take(sizeof(double) * 3 * (size_t)B);
    M.oRead = take(sizeof(double) * (1 + (size_t)B));
    M.oGd = take(sizeof(double) * B);
    M.oGmax = take(sizeof(double) * B);
    M.oGg = take(sizeof(double) * B);
    M.oSy = take(sizeof(double) * B);
    M.oYy = take(sizeof(double) * B);
    M.oUse = take(sizeof(int) * B);
    M.oKeep = take(sizeof(int) * B);
    M.oAcc = take(sizeof(int) * B);
    M.oStop = take(sizeof(int) * B);
    M.oSearch = take(sizeof(int) * B);
    M.oDone = take(sizeof(int) * B);
    M.oHdr = take(sizeof(long long) * 4);
    M.total = off;
    return M;
}

struct LCtx {
    LMap M;
    char* base;
    cudaStream_t st;
    float* vec(size_t o) const { return reinterpret_cast<float*>(base + o); }
    double* dbl(size_t o) const { return reinterpret_cast<double*>(base + o); }
    float* S(int i) const { return vec(M.oS) + (size_t)i * M.N * M.B; }
    float* Y(int i) const { return vec(M.oY) + (size_t)i * M.N * M.B; }
};

#define L_TRY(x)                                                 \
    do {                                                         \
        if ((x) != cudaSuccess) return META_ERR_CUDA;            \
    } while (0)

// out[b] = a[b] . b[b]  (b NULL with MAX: max |a[b]|)
template <bool MAX>
meta_status ldot(const LCtx& c, const float* a, const float* b, double* out) {
    k_ldot<MAX><<<dim3(c.M.nb, c.M.B), kLT, 0, c.st>>>(c.M.N, a, b, c.dbl(c.M.oPart));
    k_lred<MAX><<<c.M.B, kLT, 0, c.st>>>(c.M.nb, c.dbl(c.M.oPart), out);
    L_TRY(cudaGetLastError());
    return META_OK;
}

// d = -H g by the two-loop recursion over h stored pairs, the newest in ring
// slot head - 1.
meta_status two_loop(const LCtx& c, const float* g, float* d, int h, int head) {
    const LMap& M = c.M;
    const dim3 vg = vec_grid(M.N, M.B);
    L_TRY(cudaMemcpyAsync(d, g, sizeof(float) * (size_t)M.N * M.B, cudaMemcpyDeviceToDevice,
                          c.st));
    double* rho = c.dbl(M.oRho);
    double* alpha = c.dbl(M.oAlpha);
    const int cb = (M.B + 127) / 128;
    for (int j = 0; j < h; ++j) {  // newest first
        const int i = ((head - 1 - j) % M.m + M.m) % M.m;
        meta_status s = ldot<false>(c, c.S(i), d, c.dbl(M.oDot));
        if (s != META_OK) return s;
        k_lcoef<<<cb, 128, 0, c.st>>>(M.B, 0, rho + (size_t)i * M.B, alpha + (size_t)i * M.B,
                                      c.dbl(M.oDot), c.dbl(M.oCoef));
        k_laxpy<<<vg, kLT, 0, c.st>>>(M.N, c.dbl(M.oCoef), c.Y(i), d);
    }
    k_lscale<<<vg, kLT, 0, c.st>>>(M.N, c.dbl(M.oGamma), d);
    for (int j = h - 1; j >= 0; --j) {  // oldest first
        const int i = ((head - 1 - j) % M.m + M.m) % M.m;
        meta_status s = ldot<false>(c, c.Y(i), d, c.dbl(M.oDot));
        if (s != META_OK) return s;
        k_lcoef<<<cb, 128, 0, c.st>>>(M.B, 1, rho + (size_t)i * M.B, alpha + (size_t)i * M.B,
                                      c.dbl(M.oDot), c.dbl(M.oCoef));
        k_laxpy<<<vg, kLT, 0, c.st>>>(M.N, c.dbl(M.oCoef), c.S(i), d);
    }
    k_lneg<<<vg, kLT, 0, c.st>>>(M.N, M.B, d);
    L_TRY(cudaGetLastError());
    return META_OK;
}

meta_status lsetup(const meta_problem* prob, int m, void* lws, size_t lws_bytes, void* stream,
                   LCtx* c) {
    size_t need = 0;
    meta_status s = meta_lbfgs_workspace_size(prob, m, &need);
    if (s != META_OK) return s;
    if (!lws || (reinterpret_cast<uintptr_t>(lws) % 256) != 0 || lws_bytes < need)
        return META_ERR_WORKSPACE;
    long long N = 1;
    for (int a = 0; a < prob->ndim; ++a) N *= prob->dims[a];
    c->M = lbfgs_map(N, prob->batch, m);
    c->base = static_cast<char*>(lws);
    c->st = static_cast<cudaStream_t>(stream);
    return META_OK;
}

// Host image of a minimiser state (meta_lbfgs_state_save / _load): this
// header, then the regions of state_regions in their order.  Integers are
// little-endian, as on every machine the library builds for.
struct LStateFile {
    char magic[8];  // "METALBFS"
    uint32_t version;
    int32_t ndim, dims[3], batch, m;
    int32_t k, h, head;  // iterations done, pairs held, ring slot of the next pair
    int32_t pad[2];      // zero
    uint64_t n;         // voxels per instance
    uint64_t payload;   // bytes after the header
    uint64_t checksum;  // FNV-1a (64-bit) of the payload bytes
};
static_assert(sizeof(LStateFile) == 80 && offsetof(LStateFile, n) == 56,
              "state header layout: no implicit padding");
constexpr char kStateTag[8] = {'M', 'E', 'T', 'A', 'L', 'B', 'F', 'S'};
constexpr uint32_t kStateVersion = 1;

struct LRegion {
    size_t off, bytes;  // offset in the workspace, size
};

// What a run continues from: x's gradient g, the pair rings S and Y (all m
// slots), each pair's rho, gamma, the cost L, and the stopped / done flags.
int state_regions(const LMap& M, LRegion* r) {
    const size_t vb = sizeof(float) * (size_t)M.N * M.B;
    int n = 0;
    r[n++] = {M.oG, vb};
    r[n++] = {M.oS, vb * M.m};
    r[n++] = {M.oY, vb * M.m};
    r[n++] = {M.oRho, sizeof(double) * (size_t)M.m * M.B};
    r[n++] = {M.oGamma, sizeof(double) * M.B};
    r[n++] = {M.oRead + sizeof(double), sizeof(double) * M.B};
    r[n++] = {M.oStop, sizeof(int) * M.B};
    r[n++] = {M.oDone, sizeof(int) * M.B};
    return n;
}

size_t state_payload(const LMap& M) {
    LRegion r[8];
    const int n = state_regions(M, r);
    size_t t = 0;
    for (int i = 0; i < n; ++i) t += r[i].bytes;
    return t;
}

// FNV-1a, 64-bit (offset basis 14695981039346656037, prime 1099511628211)
uint64_t fnv1a64(const unsigned char* p, size_t n) {
    uint64_t h = 14695981039346656037ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace
}  // namespace meta

using namespace meta;

extern "C" {

meta_status meta_lbfgs_workspace_size(const meta_problem* prob, int m, size_t* bytes) {
    if (!bytes || m < 1 || m > 64) return META_ERR_INVALID_ARG;
    size_t ws = 0;
    const meta_status s = meta_workspace_size(prob, &ws);  // validates prob
    if (s != META_OK) return s;
    long long N = 1;
    for (int a = 0; a < prob->ndim; ++a) N *= prob->dims[a];
    *bytes = lbfgs_map(N, prob->batch, m).total;
    return META_OK;
}

meta_status meta_lbfgs_direction(const meta_problem* prob, int m, int npairs,
                                 const float* const* s, const float* const* y, const float* g,
                                 float* d, void* lws, size_t lws_bytes, void* stream) {
    if (!g || !d || npairs < 0 || npairs > m || (npairs > 0 && (!s || !y)))
        return META_ERR_INVALID_ARG;
    LCtx c;
    meta_status st = lsetup(prob, m, lws, lws_bytes, stream, &c);
    if (st != META_OK) return st;
    const LMap& M = c.M;
    const size_t vbytes = sizeof(float) * (size_t)M.N * M.B;
    std::vector<double> rho((size_t)M.m * M.B, 0.0), gamma(M.B, 1.0), sy(M.B), yy(M.B);
    for (int i = 0; i < npairs; ++i) {
        if (!s[i] || !y[i]) return META_ERR_INVALID_ARG;
        L_TRY(cudaMemcpyAsync(c.S(i), s[i], vbytes, cudaMemcpyDeviceToDevice, c.st));
        L_TRY(cudaMemcpyAsync(c.Y(i), y[i], vbytes, cudaMemcpyDeviceToDevice, c.st));
        st = ldot<false>(c, c.S(i), c.Y(i), c.dbl(M.oDot));
        if (st != META_OK) return st;
        L_TRY(cudaMemcpyAsync(sy.data(), c.dbl(M.oDot), sizeof(double) * M.B,
                              cudaMemcpyDeviceToHost, c.st));
        st = ldot<false>(c, c.Y(i), c.Y(i), c.dbl(M.oDot));
        if (st != META_OK) return st;
        L_TRY(cudaMemcpyAsync(yy.data(), c.dbl(M.oDot), sizeof(double) * M.B,
                              cudaMemcpyDeviceToHost, c.st));
        L_TRY(cudaStreamSynchronize(c.st));
        for (int b = 0; b < M.B; ++b) {
            const bool ok = sy[b] > 1e-12 * yy[b] && yy[b] > 0.0;
            rho[(size_t)i * M.B + b] = ok ? 1.0 / sy[b] : 0.0;
            if (ok) gamma[b] = sy[b] / yy[b];
        }
    }
    L_TRY(cudaMemcpyAsync(c.dbl(M.oRho), rho.data(), sizeof(double) * rho.size(),
                          cudaMemcpyHostToDevice, c.st));
    L_TRY(cudaMemcpyAsync(c.dbl(M.oGamma), gamma.data(), sizeof(double) * M.B,
                          cudaMemcpyHostToDevice, c.st));
    return two_loop(c, g, d, npairs, npairs % M.m);
}

// The minimiser of meta_lbfgs_minimize; with `resume` it continues from the
// state that a previous run (or meta_lbfgs_state_load) left in lws instead of
// starting at p0 with no pairs.
static meta_status lbfgs_run(const meta_problem* prob, const float* I0, const float* J,
                             float* p0, const float* mu, const float* rho, const float* lambda,
                             int iters, int m, float h0, void* ws, size_t ws_bytes, void* lws,
                             size_t lws_bytes, double* cost_hist, int* iters_done, void* stream,
                             bool resume) {
    if (!I0 || !J || !p0 || !mu || !rho || !lambda || iters < 0 || !(h0 > 0.f))
        return META_ERR_INVALID_ARG;
    LCtx c;
    meta_status st = lsetup(prob, m, lws, lws_bytes, stream, &c);
    if (st != META_OK) return st;
    const LMap& M = c.M;
    const int B = M.B;
    const size_t vbytes = sizeof(float) * (size_t)M.N * B;
    const dim3 vg = vec_grid(M.N, B);
    const int ib = (B + 127) / 128;  // blocks of the per-instance kernels
    constexpr double kC1 = 1e-4;     // Armijo constant
    constexpr int kHalvings = 12;    // backtracking steps per line search
    float* g = c.vec(M.oG);
    float* gt = c.vec(M.oGt);
    float* xt = c.vec(M.oXt);
    float* xa = c.vec(M.oXa);
    float* ga = c.vec(M.oGa);
    float* d = c.vec(M.oD);
    auto ip = [&](size_t o) { return reinterpret_cast<int*>(c.base + o); };
    LSt S;
    S.any = reinterpret_cast<unsigned long long*>(c.base + M.oRead);
    S.L = c.dbl(M.oRead) + 1;
    S.gd = c.dbl(M.oGd);
    S.gmax = c.dbl(M.oGmax);
    S.gg = c.dbl(M.oGg);
    S.step = c.dbl(M.oStep);
    S.coef = c.dbl(M.oCoef);
    S.sy = c.dbl(M.oSy);
    S.yy = c.dbl(M.oYy);
    S.rho = c.dbl(M.oRho);
    S.gamma = c.dbl(M.oGamma);
    S.cost = c.dbl(M.oCost);
    S.use = ip(M.oUse);
    S.keep = ip(M.oKeep);
    S.accepted = ip(M.oAcc);
    S.stopped = ip(M.oStop);
    S.searching = ip(M.oSearch);
    S.done = ip(M.oDone);
    // The host reads one block per line-search trial: the count of instances
    // still searching and the costs L (which also give the cost history).
    std::vector<double> rd(1 + (size_t)B);
    auto read_block = [&](unsigned long long* any) -> meta_status {
        L_TRY(cudaMemcpyAsync(rd.data(), c.dbl(M.oRead), sizeof(double) * (1 + (size_t)B),
                              cudaMemcpyDeviceToHost, c.st));
        L_TRY(cudaStreamSynchronize(c.st));
        std::memcpy(any, rd.data(), sizeof(unsigned long long));
        return META_OK;
    };
#define L_DO(x)                         \
    do {                                \
        const meta_status _s = (x);     \
        if (_s != META_OK) return _s;   \
    } while (0)

    // the state header: valid only after a run ends (or a state is loaded)
    long long hdr[4] = {0, 0, 0, 0};
    int k0 = 0, h = 0, head = 0;
    if (resume) {
        L_TRY(cudaMemcpyAsync(hdr, c.base + M.oHdr, sizeof(hdr), cudaMemcpyDeviceToHost, c.st));
        L_TRY(cudaStreamSynchronize(c.st));
        if (hdr[0] != kStateMagic || hdr[1] < 0 || hdr[1] > (long long)INT_MAX - iters ||
            hdr[2] < 0 || hdr[2] > M.m || hdr[3] < 0 || hdr[3] >= M.m)
            return META_ERR_FORMAT;
        k0 = (int)hdr[1];
        h = (int)hdr[2];
        head = (int)hdr[3];
    }
    L_TRY(cudaMemsetAsync(c.base + M.oHdr, 0, sizeof(hdr), c.st));
    if (!resume) {
        L_TRY(cudaMemsetAsync(S.rho, 0, sizeof(double) * (size_t)M.m * B, c.st));
        L_DO(meta_cost_and_grad(prob, I0, J, p0, mu, rho, lambda, S.cost, g, ws, ws_bytes, c.st));
        k_linit<<<ib, 128, 0, c.st>>>(B, S);
        L_TRY(cudaGetLastError());
    }
    if (h == 0) L_TRY(cudaMemsetAsync(d, 0, vbytes, c.st));
    unsigned long long any = 0;
    if (cost_hist) {
        L_DO(read_block(&any));
        for (int b = 0; b < B; ++b) cost_hist[b] = rd[1 + b];
    }
    for (int k = 0; k < iters; ++k) {
        // direction: the two-loop recursion, or (k_ldecide) a scaled steepest-descent
        // step for an instance without a usable pair or whose direction does not descend
        if (h > 0) L_DO(two_loop(c, g, d, h, head));
        L_DO(ldot<false>(c, g, d, S.gd));
        L_DO(ldot<true>(c, g, nullptr, S.gmax));
        L_DO(ldot<false>(c, g, g, S.gg));
        k_ldecide<<<ib, 128, 0, c.st>>>(B, M.m, h0, S);
        k_lsteep<<<vg, kLT, 0, c.st>>>(M.N, S.use, S.coef, g, d);
        L_TRY(cudaGetLastError());
        // backtracking Armijo line search, per instance, decided on the device
        for (int t = 0; t <= kHalvings; ++t) {
            k_ltrial2<<<vg, kLT, 0, c.st>>>(M.N, S, p0, d, xt);
            L_TRY(cudaGetLastError());
            L_DO(meta_cost_and_grad(prob, I0, J, xt, mu, rho, lambda, S.cost, gt, ws, ws_bytes,
                                    c.st));
            L_TRY(cudaMemsetAsync(S.any, 0, sizeof(unsigned long long), c.st));
            k_larmijo<<<ib, 128, 0, c.st>>>(B, kC1, S);
            k_lkeep<<<vg, kLT, 0, c.st>>>(M.N, S.keep, xt, gt, xa, ga);
            L_TRY(cudaGetLastError());
            L_DO(read_block(&any));  // the one host read of a trial
            if (!any) break;
        }
        k_lfinish<<<ib, 128, 0, c.st>>>(B, S);
        // new pair (s, y) of the instances that moved; x and g advance
        k_lpair<<<vg, kLT, 0, c.st>>>(M.N, S.accepted, p0, g, xa, ga, c.S(head), c.Y(head));
        L_TRY(cudaGetLastError());
        L_DO(ldot<false>(c, c.S(head), c.Y(head), S.sy));
        L_DO(ldot<false>(c, c.Y(head), c.Y(head), S.yy));
        k_lrho<<<ib, 128, 0, c.st>>>(B, head, k0 + k, S);
        L_TRY(cudaGetLastError());
        head = (head + 1) % M.m;
        h = h < M.m ? h + 1 : M.m;
        if (cost_hist)  // L of every instance as of the last trial's read
            for (int b = 0; b < B; ++b) cost_hist[(size_t)(k + 1) * B + b] = rd[1 + b];
    }
    hdr[0] = kStateMagic;
    hdr[1] = (long long)k0 + iters;
    hdr[2] = h;
    hdr[3] = head;
    L_TRY(cudaMemcpyAsync(c.base + M.oHdr, hdr, sizeof(hdr), cudaMemcpyHostToDevice, c.st));
    if (iters_done)
        L_TRY(cudaMemcpyAsync(iters_done, S.done, sizeof(int) * B, cudaMemcpyDeviceToHost, c.st));
    L_TRY(cudaStreamSynchronize(c.st));  // also keeps hdr alive until its copy is done
#undef L_DO
    return META_OK;
}

meta_status meta_lbfgs_minimize(const meta_problem* prob, const float* I0, const float* J,
                                float* p0, const float* mu, const float* rho,
                                const float* lambda, int iters, int m, float h0, void* ws,
                                size_t ws_bytes, void* lws, size_t lws_bytes, double* cost_hist,
                                int* iters_done, void* stream) {
    return lbfgs_run(prob, I0, J, p0, mu, rho, lambda, iters, m, h0, ws, ws_bytes, lws,
                     lws_bytes, cost_hist, iters_done, stream, false);
}

meta_status meta_lbfgs_resume(const meta_problem* prob, const float* I0, const float* J,
                              float* p0, const float* mu, const float* rho, const float* lambda,
                              int iters, int m, float h0, void* ws, size_t ws_bytes, void* lws,
                              size_t lws_bytes, double* cost_hist, int* iters_done,
                              void* stream) {
    return lbfgs_run(prob, I0, J, p0, mu, rho, lambda, iters, m, h0, ws, ws_bytes, lws,
                     lws_bytes, cost_hist, iters_done, stream, true);
}


meta_status meta_lbfgs_state_size(const meta_problem* prob, int m, size_t* bytes) {
    size_t lb = 0;
    const meta_status s = meta_lbfgs_workspace_size(prob, m, &lb);  // validates prob, m
    if (s != META_OK) return s;
    long long N = 1;
    for (int a = 0; a < prob->ndim; ++a) N *= prob->dims[a];
    *bytes = sizeof(LStateFile) + state_payload(lbfgs_map(N, prob->batch, m));
    return META_OK;
}

meta_status meta_lbfgs_state_check(const meta_problem* prob, int m, const void* host,
                                   size_t host_bytes) {
    size_t need = 0;
    meta_status s = meta_lbfgs_state_size(prob, m, &need);
    if (s != META_OK) return s;
    if (!host) return META_ERR_INVALID_ARG;
    if (host_bytes != need) return META_ERR_FORMAT;
    LStateFile f;
    std::memcpy(&f, host, sizeof(f));
    if (std::memcmp(f.magic, kStateTag, 8) != 0 || f.version != kStateVersion)
        return META_ERR_FORMAT;
    long long N = 1;
    for (int a = 0; a < prob->ndim; ++a) N *= prob->dims[a];
    bool same = f.ndim == prob->ndim && f.batch == prob->batch && f.m == m &&
                f.n == (uint64_t)N && f.payload == need - sizeof(LStateFile) && f.pad[0] == 0 &&
                f.pad[1] == 0;
    for (int a = 0; a < 3; ++a)
        same = same && f.dims[a] == (a < prob->ndim ? prob->dims[a] : 0);
    if (!same || f.k < 0 || f.h < 0 || f.h > m || f.head < 0 || f.head >= m)
        return META_ERR_FORMAT;
    const unsigned char* pay = static_cast<const unsigned char*>(host) + sizeof(LStateFile);
    if (fnv1a64(pay, f.payload) != f.checksum) return META_ERR_FORMAT;
    return META_OK;
}

meta_status meta_lbfgs_state_save(const meta_problem* prob, int m, const void* lws,
                                  size_t lws_bytes, void* host, size_t host_bytes,
                                  void* stream) {
    size_t need = 0;
    meta_status s = meta_lbfgs_state_size(prob, m, &need);
    if (s != META_OK) return s;
    if (!host || host_bytes < need) return META_ERR_INVALID_ARG;
    LCtx c;
    s = lsetup(prob, m, const_cast<void*>(lws), lws_bytes, stream, &c);
    if (s != META_OK) return s;
    const LMap& M = c.M;
    long long hdr[4];
    L_TRY(cudaMemcpyAsync(hdr, c.base + M.oHdr, sizeof(hdr), cudaMemcpyDeviceToHost, c.st));
    L_TRY(cudaStreamSynchronize(c.st));
    if (hdr[0] != kStateMagic) return META_ERR_FORMAT;  // no finished run in lws
    unsigned char* out = static_cast<unsigned char*>(host);
    LRegion r[8];
    const int nr = state_regions(M, r);
    size_t at = sizeof(LStateFile);
    for (int i = 0; i < nr; ++i) {
        L_TRY(cudaMemcpyAsync(out + at, c.base + r[i].off, r[i].bytes, cudaMemcpyDeviceToHost,
                              c.st));
        at += r[i].bytes;
    }
    L_TRY(cudaStreamSynchronize(c.st));
    LStateFile f;
    std::memset(&f, 0, sizeof(f));
    std::memcpy(f.magic, kStateTag, 8);
    f.version = kStateVersion;
    f.ndim = prob->ndim;
    for (int a = 0; a < prob->ndim; ++a) f.dims[a] = prob->dims[a];
    f.batch = prob->batch;
    f.m = m;
    f.k = (int32_t)hdr[1];
    f.h = (int32_t)hdr[2];
    f.head = (int32_t)hdr[3];
    f.n = (uint64_t)M.N;
    f.payload = need - sizeof(LStateFile);
    f.checksum = fnv1a64(out + sizeof(LStateFile), f.payload);
    std::memcpy(out, &f, sizeof(f));
    return META_OK;
}

meta_status meta_lbfgs_state_load(const meta_problem* prob, int m, const void* host,
                                  size_t host_bytes, void* lws, size_t lws_bytes,
                                  void* stream) {
    meta_status s = meta_lbfgs_state_check(prob, m, host, host_bytes);
    if (s != META_OK) return s;
    LCtx c;
    s = lsetup(prob, m, lws, lws_bytes, stream, &c);
    if (s != META_OK) return s;
    const LMap& M = c.M;
    LStateFile f;
    std::memcpy(&f, host, sizeof(f));
    const unsigned char* in = static_cast<const unsigned char*>(host);
    LRegion r[8];
    const int nr = state_regions(M, r);
    size_t at = sizeof(LStateFile);
    for (int i = 0; i < nr; ++i) {
        L_TRY(cudaMemcpyAsync(c.base + r[i].off, in + at, r[i].bytes, cudaMemcpyHostToDevice,
                              c.st));
        at += r[i].bytes;
    }
    const long long hdr[4] = {kStateMagic, f.k, f.h, f.head};
    L_TRY(cudaMemcpyAsync(c.base + M.oHdr, hdr, sizeof(hdr), cudaMemcpyHostToDevice, c.st));
    L_TRY(cudaStreamSynchronize(c.st));  // the host buffers may go once this returns
    return META_OK;
}

meta_status meta_gd_minimize(const meta_problem* prob, const float* I0, const float* J,
                             float* p0, const float* mu, const float* rho, const float* lambda,
                             int iters, float h0, void* ws, size_t ws_bytes, void* lws,
                             size_t lws_bytes, double* cost_hist, void* stream) {
    if (!I0 || !J || !p0 || !mu || !rho || !lambda || iters < 0 || !(h0 > 0.f))
        return META_ERR_INVALID_ARG;
    LCtx c;
    meta_status st = lsetup(prob, 1, lws, lws_bytes, stream, &c);
    if (st != META_OK) return st;
    const LMap& M = c.M;
    const int B = M.B;
    const dim3 vg = vec_grid(M.N, B);
    const int ib = (B + 127) / 128;
    float* g = c.vec(M.oG);
    double* cost = c.dbl(M.oCost);
    std::vector<double> tri(3 * (size_t)B);
    for (int k = 0; k <= iters; ++k) {
        st = meta_cost_and_grad(prob, I0, J, p0, mu, rho, lambda, cost, g, ws, ws_bytes, c.st);
        if (st != META_OK) return st;
        if (cost_hist) {  // the cost of iterate k (the host's one read per iteration)
            L_TRY(cudaMemcpyAsync(tri.data(), cost, sizeof(double) * 3 * B,
                                  cudaMemcpyDeviceToHost, c.st));
            L_TRY(cudaStreamSynchronize(c.st));
            for (int b = 0; b < B; ++b)
                cost_hist[(size_t)k * B + b] = tri[3 * b] + tri[3 * b + 1] + tri[3 * b + 2];
        }
        if (k == iters) break;
        st = ldot<true>(c, g, nullptr, c.dbl(M.oGmax));
        if (st != META_OK) return st;
        k_lgdcoef<<<ib, 128, 0, c.st>>>(B, h0, c.dbl(M.oGmax), c.dbl(M.oCoef));
        k_laxpy<<<vg, kLT, 0, c.st>>>(M.N, c.dbl(M.oCoef), g, p0);
        L_TRY(cudaGetLastError());
    }
    L_TRY(cudaStreamSynchronize(c.st));
    return META_OK;
}

}  // extern "C"
