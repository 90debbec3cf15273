// meta_api.cu -- the C ABI of include/meta.h: argument validation, workspace
// layout, Gaussian tap tables, TMA tensor maps and the launch sequence of the
// forward shooting, the cost and the discrete adjoint (arXiv:2106.08817,
// Eq. 3-4 and Sec. 2.3).  Host code only; it never allocates device memory.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "meta.h"
#include "meta_kernels.h"

#include <map>

#include <nvtx3/nvToolsExt.h>
#include <tuple>

namespace meta {
namespace {

constexpr size_t kAlign = 256;

// Process-wide tile shapes per problem shape (meta_autotune / meta_tuning_set).
using TuneKey = std::tuple<int, int, int, int, int, uint32_t>;
std::mutex g_tune_mu;
std::map<TuneKey, meta_tuning> g_tune;

TuneKey tune_key(const meta_problem* pr) {
    uint32_t sb;
    std::memcpy(&sb, &pr->sigma, 4);
    return TuneKey(pr->ndim, pr->dims[0], pr->ndim == 3 ? pr->dims[1] : 0,
                   pr->dims[pr->ndim - 1], pr->batch, sb);
}

bool find_tuning(const meta_problem* pr, meta_tuning* t) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(pr));
    if (it == g_tune.end()) return false;
    *t = it->second;
    return true;
}

constexpr int kMaxSplit = 16;  // largest batch split of a recorded plan

// Sub-batch k of a batch split into S: instances [first, first + count).
void split_range(int B, int S, int k, int* first, int* count) {
    const int q = B / S, r = B % S;
    *first = k * q + (k < r ? k : r);
    *count = q + (k < r ? 1 : 0);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Workspace map (byte offsets from the workspace base).
struct Layout {
    Geom g;
    int ndim, T, nblk;
    int k;        // checkpoint stride; 0 = every state kept (slot = time)
    int pdet;     // momentum update p~ det(Id - dt Dv) (else p~ (1 - dt div v))
    int scheme;   // META_SCHEME_SL / _EULER / _HYBRID
    int nseg;     // segments of k steps (k > 0)
    int nbuf;     // sets of segment slots (k > 0): 2 where that still saves memory, else 1
    int nstate;   // state slots
    int nu;       // u slots
    size_t off_fault, off_maxdisp, off_partials;
    size_t off_states, off_u, off_SA, off_SB, off_SV;
    size_t off_REC, off_IHP, off_PHP, off_RAW;
    size_t total;

    // Keeping every state: slot = time.  With stride k: state t of segment s
    // (t in [s k, s k + k]) lives in checkpoint slot s when t = s k, else in
    // segment slot nseg + (s % nbuf) k + (t - s k) - 1: nbuf sets of k segment
    // slots, taken by the segments in turn, so that the forward leaves its last
    // nbuf segments in place; u_t (t > 0) in slot ((t / k) % nbuf) k + t % k, u_0 in
    // slot nbuf k.
    int state_slot(int t, int s) const {
        if (k == 0) return t;
        return t == s * k ? s : nseg + (s % nbuf) * k + (t - s * k) - 1;
    }
    int u_slot(int t) const {
        return k == 0 ? t : (t == 0 ? nbuf * k : ((t / k) % nbuf) * k + t % k);
    }
    int seg_of(int t) const { return k == 0 ? 0 : t / k; }
    // Segments the adjoint re-runs from their checkpoints: all but the last nbuf.
    bool recomputed(int s) const { return k != 0 && s < seg_of(T - 1) - (nbuf - 1); }
    int seg_end(int s) const { return k == 0 ? T : (s * k + k < T ? s * k + k : T); }
    // slot written by the first forward pass for time t + 1
    int forward_out_slot(int t) const {
        if (k == 0) return t + 1;
        if ((t + 1) % k == 0 && t + 1 < T) return (t + 1) / k;  // next checkpoint
        return state_slot(t + 1, t / k);
    }
    int final_slot() const { return k == 0 ? T : state_slot(T, (T - 1) / k); }
};

meta_status validate(const meta_problem* pr) {
    if (!pr) return META_ERR_INVALID_ARG;
    if (pr->ndim != 2 && pr->ndim != 3) return META_ERR_INVALID_ARG;
    if (pr->batch < 1 || pr->batch > 16384) return META_ERR_INVALID_ARG;
    if (pr->T < 1 || pr->T > 4096) return META_ERR_INVALID_ARG;
    if (!(pr->sigma > 0.f) || !(pr->sigma <= 18.f)) return META_ERR_INVALID_ARG;
    if (pr->ckpt_stride < 0 || pr->ckpt_stride > 4096) return META_ERR_INVALID_ARG;
    if (pr->p_update != META_P_UPDATE_DIV && pr->p_update != META_P_UPDATE_DET)
        return META_ERR_INVALID_ARG;
    if (pr->scheme != META_SCHEME_SL && pr->scheme != META_SCHEME_EULER &&
        pr->scheme != META_SCHEME_HYBRID)
        return META_ERR_INVALID_ARG;
    if (pr->scheme != META_SCHEME_SL && pr->p_update != META_P_UPDATE_DIV)
        return META_ERR_INVALID_ARG;
    for (int a = 0; a < pr->ndim; ++a)
        if (pr->dims[a] < 2 || pr->dims[a] > 65536) return META_ERR_SHAPE;
    if (pr->ndim == 3) {
        // x-pass grid.y = ceil(ny/4) * ceil(nz/4); strided grids = tiles * extent
        const long long gy = (long long)((pr->dims[1] + 3) / 4) * ((pr->dims[0] + 3) / 4);
        const long long gy1 = (long long)((pr->dims[1] + kTA - 1) / kTA) * pr->dims[0];
        const long long gy0 = (long long)((pr->dims[0] + kTA - 1) / kTA) * pr->dims[1];
        const long long gp = (long long)((pr->dims[1] + 7) / 8) * pr->dims[0];
        const long long gg = (long long)((pr->dims[1] + 3) / 4) * ((pr->dims[0] + 1) / 2);
        if (gy > 65535 || gy1 > 65535 || gy0 > 65535 || gp > 65535 || gg > 65535)
            return META_ERR_SHAPE;
    } else {
        if ((pr->dims[0] + 7) / 8 > 65535) return META_ERR_SHAPE;
    }
    return META_OK;
}

Layout make_layout(const meta_problem* pr) {
    Layout L;
    std::memset(&L, 0, sizeof(L));
    const int d = pr->ndim;
    L.ndim = d;
    L.T = pr->T;
    L.pdet = pr->p_update == META_P_UPDATE_DET ? 1 : 0;
    L.scheme = pr->scheme;
    Geom& g = L.g;
    g.nz = d == 3 ? pr->dims[0] : 1;
    g.ny = pr->dims[d - 2];
    g.nx = pr->dims[d - 1];
    g.P = (g.nx + 3) / 4 * 4;
    g.slab = (long long)g.ny * g.P;
    g.inst = (long long)g.nz * g.slab;
    g.B = pr->batch;
    g.nT = pr->T;
    g.txw = even_tile(g.nx, kTX, kBX);
    g.ly = even_tile(g.ny, kTA, kBA);
    g.lz = d == 3 ? even_tile(g.nz, kTA, kBA) : kBA;
    g.zct = g.zca = 0;
    g.chk = nullptr;  // set to the workspace status word by setup
    {
        const unsigned long long nyt = (unsigned long long)(g.ny + 7) / 8;
        g.nyt_mul = nyt == 1 ? 0u : (unsigned)(((1ull << 32) + nyt - 1) / nyt);
    }
    meta_tuning tn;
    if (find_tuning(pr, &tn)) {
        if (tn.txw > 0) g.txw = tn.txw;
        if (tn.ly > 0) g.ly = tn.ly;
        if (d == 3 && tn.lz > 0) g.lz = tn.lz;
        if (d == 3) {
            g.zct = tn.zc_transport;
            g.zca = tn.zc_advect;
        }
    }
    // a stride of 0, 1 or >= T keeps every state
    L.k = (pr->ckpt_stride > 1 && pr->ckpt_stride < pr->T) ? pr->ckpt_stride : 0;
    L.nseg = L.k ? (pr->T + L.k - 1) / L.k : 1;
    // two sets of segment slots (the last two segments need no recompute) where
    // that layout is still smaller than keeping every state, else one
    L.nbuf = 1;
    if (L.k && 2 * (L.nseg + 2 * L.k) + d * (2 * L.k + 1) < 2 * (pr->T + 1) + d * pr->T)
        L.nbuf = 2;
    L.nstate = L.k ? L.nseg + L.nbuf * L.k : pr->T + 1;
    L.nu = L.k ? L.nbuf * L.k + 1 : pr->T;
    // cost partial sums: one CTA of 8 warps per 8 rows, at most 1024 per instance (a
    // 3-D volume's CTAs take several rows per warp, and the final sum reads fewer)
    long long nblk = ((long long)g.nz * g.ny + 7) / 8;
    if (nblk < 1) nblk = 1;
    if (nblk > 1024) nblk = 1024;
    L.nblk = (int)nblk;

    const size_t fslice = (size_t)g.inst * 4;  // bytes of one pitched field
    const size_t B = (size_t)g.B;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    };
    L.off_fault = take(16);
    L.off_maxdisp = take(sizeof(unsigned int) * kMaxdispStride * (size_t)pr->T * B);
    L.off_partials = take(sizeof(double) * 3 * B * (size_t)L.nblk);
    L.off_states = take(fslice * 2 * B * (size_t)L.nstate);
    L.off_u = take(fslice * (size_t)d * B * (size_t)L.nu);
    L.off_SA = take(fslice * (size_t)d * B);
    L.off_SB = take(fslice * (size_t)d * B);
    L.off_SV = take(fslice * (size_t)d * B);
    L.off_REC = take(fslice * (size_t)(d + 4) * B);
    L.off_IHP = take(fslice * B);
    L.off_PHP = take(fslice * B);
    // raw I^, p^ of every step (Eulerian, hybrid)
    L.off_RAW = L.scheme != META_SCHEME_SL ? take(fslice * 2 * B) : 0;
    L.total = off;
    return L;
}

// Gaussian taps of K: exp(-k^2 / (2 sigma^2)), |k| <= r = ceil(3 sigma),
// normalised to sum 1 in double and rounded to float.
//  xpass:   w[k'] = tap(k' - r4) for k' in [r4 - r, r4 + r], 0 elsewhere,
//           kp = roundup(r4 + r + 1, 8)   (window starts r4 left of the output)
//  strided: w[k']  = tap(k' - r) for k' in [0, 2r], kp = roundup(2r + 1, 8)
// Radius of the x pass's staged halo: r = ceil(3 sigma) rounded up to 4.
int xpass_r(float sigma) { return (int)std::ceil(3.0 * (double)sigma); }
int xpass_r4(float sigma) { return (xpass_r(sigma) + 3) / 4 * 4; }
// Taps in the strided passes' loop: roundup(2r + 1, 8) (the TMA box holds L + kp rows).
int strided_kp(float sigma) { return (2 * xpass_r(sigma) + 1 + 7) / 8 * 8; }

void make_taps(float sigma, Taps* xpass, Taps* strided) {
    const int r = (int)std::ceil(3.0 * (double)sigma);
    double t[2 * kMaxR + 1];
    double Z = 0.0;
    for (int k = -r; k <= r; ++k) {
        t[k + r] = std::exp(-(double)k * (double)k / (2.0 * (double)sigma * (double)sigma));
        Z += t[k + r];
    }
    const int r4 = (r + 3) / 4 * 4;
    std::memset(xpass, 0, sizeof(Taps));
    std::memset(strided, 0, sizeof(Taps));
    xpass->r = strided->r = r;
    xpass->r4 = strided->r4 = r4;
    xpass->kp = (r4 + r + 1 + 7) / 8 * 8;
    strided->kp = (2 * r + 1 + 7) / 8 * 8;
    for (int k = -r; k <= r; ++k) {
        xpass->w[r4 + k] = (float)(t[k + r] / Z);
        strided->w[r + k] = (float)(t[k + r] / Z);
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor map over `nslices` pitched slices starting at `base`: dims
// {nx, ny, (nz), nslices}; zero fill outside (the zero padding of K).
bool encode_map(CUtensorMap* m, const Geom& g, int ndim, void* base, int nslices, int bx,
                int by, int bz) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
    cuuint32_t rank;
    if (ndim == 2) {
        rank = 3;
        dims[0] = g.nx;
        dims[1] = g.ny;
        dims[2] = nslices;
        strides[0] = (cuuint64_t)g.P * 4;
        strides[1] = (cuuint64_t)g.inst * 4;
        box[0] = bx;
        box[1] = by;
        box[2] = 1;
    } else {
        rank = 4;
        dims[0] = g.nx;
        dims[1] = g.ny;
        dims[2] = g.nz;
        dims[3] = nslices;
        strides[0] = (cuuint64_t)g.P * 4;
        strides[1] = (cuuint64_t)g.slab * 4;
        strides[2] = (cuuint64_t)g.inst * 4;
        box[0] = bx;
        box[1] = by;
        box[2] = bz;
        box[3] = 1;
    }
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 5-D tensor map over fields of a batch of pitched instances: dims {nx, ny,
// nz, B, nfields}, field f of instance b at slice f * B + b; boxes of a 3-D
// marching kernel's plane window (40 x box_rows x 1 x 1 x box_nf); zero fill outside.
bool encode_map5(CUtensorMap* m, const Geom& g, void* base, int nfields, int box_nf,
                 int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[5] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz,
                                (cuuint64_t)g.B, (cuuint64_t)nfields};
    const cuuint64_t strides[4] = {(cuuint64_t)g.P * 4, (cuuint64_t)g.slab * 4,
                                   (cuuint64_t)g.inst * 4, (cuuint64_t)g.B * g.inst * 4};
    const cuuint32_t box[5] = {40, (cuuint32_t)box_rows, 1, 1, (cuuint32_t)box_nf};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

struct Ctx {
    Layout L;
    char* ws;
    Taps tx, ts;
    CUtensorMap tmI, tmP, tmSAy, tmSBz, tmSVx;
    CUtensorMap tmTr[3];  // 3-D transport: records 0..5, div^, (I_t, p_t)
    CUtensorMap tmAdv[2];  // 3-D advect: u (3 components), (I_t, p_t)
    cudaStream_t st;
    unsigned int* fault;
    unsigned int* maxdisp;
    double* partials;
    float *states, *u, *SA, *SB, *SV, *REC, *IHP, *PHP, *RAW;
};

// Raw p^ half of the RAW region (NULL when RAW is not allocated).
float* raw_p(const Ctx& c) { return c.RAW ? c.RAW + (size_t)c.L.g.B * c.L.g.inst : nullptr; }

meta_status map_status(cudaError_t e) { return e == cudaSuccess ? META_OK : META_ERR_CUDA; }

// Optional per-launch event timer (profiling aid; see meta_timer_start).
struct Timer {
    bool on = false;
    int cap = 0, used = 0;
    std::vector<cudaEvent_t> ev;  // 2 per launch
    std::vector<int> cls;
};
Timer g_timer;

struct Timed {
    int slot = -1;
    cudaStream_t st;
    Timed(int k, cudaStream_t s) : st(s) {
        if (g_timer.on && g_timer.used < g_timer.cap) {
            slot = g_timer.used++;
            g_timer.cls[slot] = k;
            cudaEventRecord(g_timer.ev[2 * slot], st);
        }
    }
    ~Timed() {
        if (slot >= 0) cudaEventRecord(g_timer.ev[2 * slot + 1], st);
    }
};

meta_status setup(const meta_problem* pr, void* ws, size_t ws_bytes, void* stream, Ctx* c) {
    meta_status s = validate(pr);
    if (s != META_OK) return s;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return META_ERR_WORKSPACE;
    c->L = make_layout(pr);
    if (ws_bytes < c->L.total) return META_ERR_WORKSPACE;
    c->ws = static_cast<char*>(ws);
    c->st = static_cast<cudaStream_t>(stream);
    const Layout& L = c->L;
    c->fault = reinterpret_cast<unsigned int*>(c->ws + L.off_fault);
    c->L.g.chk = c->fault;
    c->maxdisp = reinterpret_cast<unsigned int*>(c->ws + L.off_maxdisp);
    c->partials = reinterpret_cast<double*>(c->ws + L.off_partials);
    auto F = [&](size_t off) { return reinterpret_cast<float*>(c->ws + off); };
    c->states = F(L.off_states);
    c->u = F(L.off_u);
    c->SA = F(L.off_SA);
    c->SB = F(L.off_SB);
    c->SV = F(L.off_SV);
    c->REC = F(L.off_REC);
    c->RAW = L.off_RAW ? F(L.off_RAW) : nullptr;
    c->IHP = F(L.off_IHP);
    c->PHP = F(L.off_PHP);
    make_taps(pr->sigma, &c->tx, &c->ts);
    const Geom& g = L.g;
    const int d = L.ndim, B = g.B;
    const int LW = xpass_lw(g.txw, c->tx.r, c->tx.r4);
    const int nst = 2 * B * L.nstate;
    bool ok = true;
    if (d == 2) {
        ok &= encode_map(&c->tmI, g, 2, c->states, nst, LW, kRows + 2, 1);
        ok &= encode_map(&c->tmP, g, 2, c->states, nst, LW, kRows, 1);
        ok &= encode_map(&c->tmSAy, g, 2, c->SA, d * B, kTXS, g.ly + c->ts.kp, 1);
        ok &= encode_map(&c->tmSVx, g, 2, c->SV, d * B, LW, kRows, 1);
        c->tmSBz = c->tmSAy;
    } else {
        ok &= encode_map(&c->tmI, g, 3, c->states, nst, LW, 6, 6);
        ok &= encode_map(&c->tmP, g, 3, c->states, nst, LW, 4, 4);
        ok &= encode_map(&c->tmSAy, g, 3, c->SA, d * B, kTXS, g.ly + c->ts.kp, 1);
        ok &= encode_map(&c->tmSBz, g, 3, c->SB, d * B, kTXS, 1, g.lz + c->ts.kp);
        ok &= encode_map(&c->tmSVx, g, 3, c->SV, d * B, LW, 4, 4);
        ok &= encode_map5(&c->tmTr[0], g, c->REC, d + 4, 6, kTransRows + 2);
        ok &= encode_map5(&c->tmTr[1], g, c->REC, d + 4, 1, kTransRows + 2);
        ok &= encode_map5(&c->tmTr[2], g, c->states, 2 * L.nstate, 2, kTransRows + 2);
        ok &= encode_map5(&c->tmAdv[0], g, c->u, 3 * L.nu, 3, kAdvRows + 2);
        ok &= encode_map5(&c->tmAdv[1], g, c->states, 2 * L.nstate, 2, kAdvRows + 2);
    }
    return ok ? META_OK : META_ERR_UNSUPPORTED;
}

#define META_TRY(expr)                                  \
    do {                                                \
        meta_status _s = map_status(expr);              \
        if (_s != META_OK) return _s;                   \
    } while (0)

// Launch `expr` (a launcher returning cudaError_t) as kernel class k.
#define META_LAUNCH(k, st, expr)                        \
    do {                                                \
        Timed _t((k), (st));                            \
        meta_status _s = map_status(expr);              \
        if (_s != META_OK) return _s;                   \
    } while (0)

// Forward step t: m = p grad I and the blur into u slot su, then the advect
// from state slot sin to sout.
meta_status forward_step(Ctx& c, const Coefs& cf, int t, int sin, int sout, int su,
                         bool advect) {
    const Layout& L = c.L;
    const Geom& g = L.g;
    const int d = L.ndim, B = g.B;
    float* ut = c.u + (size_t)su * d * B * g.inst;
    META_LAUNCH(META_K_XPASS_M, c.st,
                launch_xpass(d, true, c.tmI, c.tmP, c.tx, g, 2 * sin * B, (2 * sin + 1) * B, c.states, 0, 0,
                             c.SA, c.fault, c.st));
    if (d == 2) {
        META_LAUNCH(META_K_STRIDED_FWD, c.st,
                    launch_strided(2, 0, c.tmSAy, c.ts, g, 0, 0, d * B, nullptr, 1.f, ut, c.fault,
                                   c.st));
    } else {
        META_LAUNCH(META_K_STRIDED_FWD, c.st,
                    launch_strided(3, 1, c.tmSAy, c.ts, g, 0, 0, d * B, nullptr, 1.f, c.SB,
                                   c.fault, c.st));
        META_LAUNCH(META_K_STRIDED_FWD, c.st,
                    launch_strided(3, 0, c.tmSBz, c.ts, g, 0, 0, d * B, nullptr, 1.f, ut, c.fault,
                                   c.st));
    }
    if (advect) {
        Slots sl{};
        sl.st = sin;
        sl.st1 = sout;
        sl.ut = su;
        if (L.scheme == META_SCHEME_SL)
            META_LAUNCH(META_K_ADVECT, c.st,
                        launch_advect(g, d, cf, t, sl, c.states, c.u, c.maxdisp, c.tmAdv, c.fault,
                                      c.st));
        else
            META_LAUNCH(META_K_EULER, c.st,
                        launch_euler(g, d, cf, t, sl, L.scheme == META_SCHEME_HYBRID, c.states,
                                     c.u, c.maxdisp, c.st));
    }
    return META_OK;
}

// Forward shooting t = 0..T-1 (the initial state is already in slot 0).  With
// wT not null it also integrates the deformation w_t = phi_t - Id, ping-ponged
// between SV and REC (neither is used by a forward pass), and sets *wT to the
// buffer that holds w_T.
// Phases of a call as NVTX ranges ("meta.cost_and_grad" around "meta.forward",
// "meta.cost", "meta.adjoint" and, inside it, one "meta.recompute" per
// re-run checkpoint segment).  They are host ranges: each brackets the
// enqueueing of its phase's kernels, which profilers (ncu --nvtx) attribute
// to it.  A host callback (meta_trace_set) sees the same pushes and pops.
std::mutex g_trace_mu;
meta_trace_fn g_trace_fn = nullptr;
void* g_trace_user = nullptr;

void trace_emit(const char* name, int push) {
    meta_trace_fn fn;
    void* user;
    {
        std::lock_guard<std::mutex> lk(g_trace_mu);
        fn = g_trace_fn;
        user = g_trace_user;
    }
    if (fn) fn(name, push, user);
}

struct Range {
    const char* name;
    explicit Range(const char* n) : name(n) {
        nvtxRangePushA(n);
        trace_emit(n, 1);
    }
    ~Range() {
        trace_emit(name, 0);
        nvtxRangePop();
    }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

meta_status run_forward(Ctx& c, const Coefs& cf, const float** wT = nullptr) {
    Range r("meta.forward");
    const Layout& L = c.L;
    const size_t md_words = (size_t)kMaxdispStride * L.T * L.g.B;
    if (std::vector<PRec>* r = recorder()) {
        PRec e{};
        e.kind = PK_ZERO;
        e.grid = dim3((unsigned)((md_words + 1023) / 1024));
        e.bx = 256;
        e.by = 1;
        e.a.md = c.maxdisp;
        e.a.n = (int)md_words;
        r->push_back(e);
    } else {
        META_TRY(cudaMemsetAsync(c.maxdisp, 0, sizeof(unsigned int) * md_words, c.st));
    }
    for (int t = 0; t < L.T; ++t) {
        const meta_status s = forward_step(c, cf, t, L.state_slot(t, L.seg_of(t)),
                                           L.forward_out_slot(t), L.u_slot(t), true);
        if (s != META_OK) return s;
        if (wT) {
            float* wout = (t & 1) ? c.REC : c.SV;
            const float* win = t == 0 ? nullptr : ((t & 1) ? c.SV : c.REC);
            META_LAUNCH(META_K_DEFORM, c.st,
                        launch_deform(L.g, L.ndim, cf, L.u_slot(t), c.u, win, wout, c.st));
            *wT = wout;
        }
    }
    return META_OK;
}

// Recomputes forward segment s from its checkpoint: the states and u of its
// steps (the segment's last state is not needed by the adjoint).
meta_status recompute_segment(Ctx& c, const Coefs& cf, int s) {
    Range r("meta.recompute");
    const Layout& L = c.L;
    const int e = L.seg_end(s);
    for (int t = s * L.k; t < e; ++t) {
        const meta_status st = forward_step(c, cf, t, L.state_slot(t, s),
                                            L.state_slot(t + 1, s), L.u_slot(t), t + 1 < e);
        if (st != META_OK) return st;
    }
    return META_OK;
}

// Slots of the cost / adjoint start: records of step T-1, states T and 0, u_0.
Slots start_slots(const Layout& L) {
    Slots sl{};
    sl.st1 = L.state_slot(L.T - 1, L.seg_of(L.T - 1));
    sl.ut1 = L.u_slot(L.T - 1);
    sl.s0 = 0;
    sl.u0 = L.u_slot(0);
    sl.sT = L.final_slot();
    return sl;
}

// Reverse sweep; REC holds the records of step T-1 on entry (from the adjoint
// start of the cost or of meta_shoot_adjoint).  mode 1: cost gradient into out0; mode 2:
// shooting adjoint into out0 / gI0.  With step checkpointing, each segment
// but the last (still in place after the forward) is recomputed from its
// checkpoint just before the gradp of the step that follows it, so that every
// gradp builds the record of the step before it directly.
meta_status run_adjoint_other(Ctx& c, const Coefs& cf, int mode, float* out0, float* gI0);

meta_status run_adjoint(Ctx& c, const Coefs& cf, int mode, float* out0, float* gI0) {
    Range r("meta.adjoint");
    if (c.L.scheme != META_SCHEME_SL) return run_adjoint_other(c, cf, mode, out0, gI0);
    const Layout& L = c.L;
    const Geom& g = L.g;
    const int d = L.ndim, B = g.B;
    float* rawI = c.RAW;
    float* rawP = c.RAW ? c.RAW + (size_t)B * g.inst : nullptr;
    for (int t = L.T - 1; t >= 0; --t) {
        const int s = L.seg_of(t);
        Slots sl{};
        sl.st = L.state_slot(t, s);
        sl.ut = L.u_slot(t);
        sl.u0 = L.u_slot(0);
        META_LAUNCH(META_K_ADJ_GATHER, c.st,
                    launch_adj_transport(g, d, cf, t, sl, c.tmTr, c.states, c.maxdisp, c.REC, c.SV, c.IHP,
                                         c.PHP, c.fault, c.st));
        if (L.pdet)
            META_LAUNCH(META_K_ADJ_JAC, c.st,
                        launch_adj_jacT(g, d, cf, sl, c.u, c.REC, c.SV, c.st));
        // m^ = K(-rho v^): x-pass SV -> SA, then the strided passes
        META_LAUNCH(META_K_XPASS_ADJ, c.st,
                    launch_xpass(d, false, c.tmSVx, c.tmSVx, c.tx, g, 0, 0, nullptr, 0, d * B, c.SA,
                                 c.fault, c.st));
        float* mh;
        if (d == 2) {
            META_LAUNCH(META_K_STRIDED_ADJ, c.st,
                        launch_strided(2, 0, c.tmSAy, c.ts, g, 0, 0, d * B, cf.rho, -1.f, c.SB,
                                       c.fault, c.st));
            mh = c.SB;
        } else {
            META_LAUNCH(META_K_STRIDED_ADJ, c.st,
                        launch_strided(3, 1, c.tmSAy, c.ts, g, 0, 0, d * B, nullptr, 1.f, c.SB,
                                       c.fault, c.st));
            META_LAUNCH(META_K_STRIDED_ADJ, c.st,
                        launch_strided(3, 0, c.tmSBz, c.ts, g, 0, 0, d * B, cf.rho, -1.f, c.SV,
                                       c.fault, c.st));
            mh = c.SV;
        }
        int m;
        if (t == 0) {
            m = mode;
        } else {
            if (L.k && t == s * L.k && L.recomputed(s - 1)) {
                // step t-1 ends segment s-1, which (unless it is one of the last two,
                // still in place) comes back from its checkpoint now, after this
                // step's transport and blur and before its gradp, which then builds
                // the record of step t-1 as in every other step (the recompute writes
                // the other parity's segment and u slots, SA and SB, none of which
                // this step still reads)
                const meta_status st = recompute_segment(c, cf, s - 1);
                if (st != META_OK) return st;
            }
            m = 0;
            sl.st1 = L.state_slot(t - 1, L.seg_of(t - 1));
            sl.ut1 = L.u_slot(t - 1);
        }
        META_LAUNCH(META_K_ADJ_GRADP, c.st,
                    launch_adj_gradp(g, d, cf, t, m, sl, c.states, c.u, c.maxdisp, mh, c.IHP,
                                     c.PHP, c.REC, rawI, rawP, out0, gI0, c.st));
    }
    return META_OK;
}

// Adjoint sweep of the Eulerian (one pointwise transpose per step) and hybrid
// schemes (its semi-Lagrangian image step through the records and the gather
// transport, then the Eulerian momentum part); both then blur v^ and run
// k_adj_gradp, which leaves the raw I^_t, p^_t in RAW for the step before
// (mode 3) or the outputs at t = 0.
meta_status run_adjoint_other(Ctx& c, const Coefs& cf, int mode, float* out0, float* gI0) {
    const Layout& L = c.L;
    const Geom& g = L.g;
    const int d = L.ndim, B = g.B;
    float* rawI = c.RAW;
    float* rawP = raw_p(c);
    for (int t = L.T - 1; t >= 0; --t) {
        const int s = L.seg_of(t);
        if (L.recomputed(s) && t == L.seg_end(s) - 1) {
            const meta_status st = recompute_segment(c, cf, s);
            if (st != META_OK) return st;
        }
        Slots sl{};
        sl.st = L.state_slot(t, s);
        sl.ut = L.u_slot(t);
        sl.u0 = L.u_slot(0);
        if (L.scheme == META_SCHEME_EULER) {
            META_LAUNCH(META_K_ADJ_GATHER, c.st,
                        launch_euler_adj(g, d, cf, sl, c.states, c.u, rawI, rawP, c.IHP, c.PHP,
                                         c.SV, c.st));
        } else {
            if (t < L.T - 1) {  // the record of step T-1 comes from the adjoint start
                Slots rs{};
                rs.st1 = sl.st;
                rs.ut1 = sl.ut;
                META_LAUNCH(META_K_ADJ_INIT, c.st,
                            launch_adj_records(g, d, cf, rs, c.states, c.u, rawI, rawP, c.REC,
                                               c.st));
            }
            META_LAUNCH(META_K_ADJ_GATHER, c.st,
                        launch_adj_transport(g, d, cf, t, sl, c.tmTr, c.states, c.maxdisp, c.REC, c.SV,
                                             c.IHP, c.PHP, c.fault, c.st));
            META_LAUNCH(META_K_ADJ_GATHER, c.st,
                        launch_hybrid_p(g, d, cf, sl, c.states, c.u, rawP, c.PHP, c.SV, c.st));
        }
        META_LAUNCH(META_K_XPASS_ADJ, c.st,
                    launch_xpass(d, false, c.tmSVx, c.tmSVx, c.tx, g, 0, 0, nullptr, 0, d * B, c.SA,
                                 c.fault, c.st));
        float* mh;
        if (d == 2) {
            META_LAUNCH(META_K_STRIDED_ADJ, c.st,
                        launch_strided(2, 0, c.tmSAy, c.ts, g, 0, 0, d * B, cf.rho, -1.f, c.SB,
                                       c.fault, c.st));
            mh = c.SB;
        } else {
            META_LAUNCH(META_K_STRIDED_ADJ, c.st,
                        launch_strided(3, 1, c.tmSAy, c.ts, g, 0, 0, d * B, nullptr, 1.f, c.SB,
                                       c.fault, c.st));
            META_LAUNCH(META_K_STRIDED_ADJ, c.st,
                        launch_strided(3, 0, c.tmSBz, c.ts, g, 0, 0, d * B, cf.rho, -1.f, c.SV,
                                       c.fault, c.st));
            mh = c.SV;
        }
        META_LAUNCH(META_K_ADJ_GRADP, c.st,
                    launch_adj_gradp(g, d, cf, t, t == 0 ? mode : 3, sl, c.states, c.u,
                                     c.maxdisp, mh, c.IHP, c.PHP, c.REC, rawI, rawP, out0, gI0,
                                     c.st));
    }
    return META_OK;
}

// Workspace bytes of a batch split into S sub-batches, each in its own
// 256-byte aligned region.
size_t split_bytes(const meta_problem* pr, int S) {
    size_t total = 0;
    for (int k = 0; k < S; ++k) {
        int first, count;
        split_range(pr->batch, S, k, &first, &count);
        meta_problem sub = *pr;
        sub.batch = count;
        total += align_up(make_layout(&sub).total, kAlign);
    }
    return total;
}

// One cost_and_grad call with an optional fault word other than the one in
// its workspace (the sub-batches of a split plan all report to the first).
// Every scheme has its adjoint; the det momentum update belongs to the
// semi-Lagrangian scheme (validate refuses the other combinations).
meta_status adjoint_scheme(const meta_problem* pr) { return validate(pr); }

meta_status cost_and_grad_impl(const meta_problem* prob, const float* I0, const float* J,
                               const float* p0, const float* mu, const float* rho,
                               const float* lambda, double* cost, float* grad, void* ws,
                               size_t ws_bytes, void* stream, unsigned int* fault) {
    if (!I0 || !J || !p0 || !mu || !rho || !lambda || !cost) return META_ERR_INVALID_ARG;
    {
        const meta_status a = adjoint_scheme(prob);
        if (a != META_OK) return a;
    }
    Range r("meta.cost_and_grad");
    Ctx c;
    meta_status s = setup(prob, ws, ws_bytes, stream, &c);
    if (s != META_OK) return s;
    if (fault) {
        c.fault = fault;
        c.L.g.chk = fault;
    }
    const Geom& g = c.L.g;
    const Coefs cf{mu, rho, lambda, 1.f / (float)c.L.T, c.L.pdet, c.L.scheme};
    META_LAUNCH(META_K_PACK, c.st,
                launch_pack(g, c.L.ndim, I0, p0, c.states, c.states + (size_t)g.B * g.inst, c.st));
    s = run_forward(c, cf);
    if (s != META_OK) return s;
    {
        Range rc("meta.cost");
        META_LAUNCH(META_K_COST, c.st,
                    launch_cost(g, c.L.ndim, cf, start_slots(c.L), c.states, c.u, J, c.maxdisp,
                                c.REC, c.IHP, c.PHP, c.RAW, raw_p(c), c.partials, c.L.nblk,
                                cost, c.st));
    }
    if (!grad) return META_OK;
    return run_adjoint(c, cf, 1, grad, nullptr);
}

}  // namespace

std::vector<PRec>*& recorder() {
    static thread_local std::vector<PRec>* r = nullptr;
    return r;
}

// The range and launch-limit checks of meta_tuning_set, without storing.
meta_status tuning_check(const meta_problem* prob, const meta_tuning* tun) {
    const meta_status s = validate(prob);
    if (s != META_OK) return s;
    if (!tun) return META_ERR_INVALID_ARG;
    const int d = prob->ndim;
    const int nz = d == 3 ? prob->dims[0] : 1, ny = prob->dims[d - 2];
    auto len_ok = [](int v, int q, int mx) { return v == 0 || (v >= q && v <= mx && v % q == 0); };
    if (!len_ok(tun->ly, kBA, kTAMax) || !len_ok(tun->lz, kBA, kTAMax) || !len_ok(tun->txw, kBX, 256))
        return META_ERR_INVALID_ARG;
    // a strided tile and its taps are staged by one TMA box (<= 256 along the axis)
    const int kp_s = strided_kp(prob->sigma);
    if (tun->ly + kp_s > 256 || tun->lz + kp_s > 256) return META_ERR_INVALID_ARG;
    // the x pass stages rows of txw + 2 hx floats by one TMA box (<= 256)
    if (tun->txw && xpass_lw(tun->txw, xpass_r(prob->sigma), xpass_r4(prob->sigma)) > kMaxLW)
        return META_ERR_INVALID_ARG;
    if (tun->zc_transport < 0 || tun->zc_transport > nz || tun->zc_advect < 0 ||
        tun->zc_advect > nz)
        return META_ERR_INVALID_ARG;
    if (d == 2 && (tun->lz != 0 || tun->zc_transport != 0 || tun->zc_advect != 0))
        return META_ERR_INVALID_ARG;
    if (tun->split < 0 || tun->split > (prob->batch < kMaxSplit ? prob->batch : kMaxSplit))
        return META_ERR_INVALID_ARG;
    // grid limits of the strided passes (y: tiles * nz, z: tiles * ny)
    if (tun->ly && (long long)((ny + tun->ly - 1) / tun->ly) * nz > 65535)
        return META_ERR_INVALID_ARG;
    if (tun->lz && (long long)((nz + tun->lz - 1) / tun->lz) * ny > 65535)
        return META_ERR_INVALID_ARG;
    return META_OK;
}

void tuning_snapshot(std::vector<TuneEntry>* out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    out->clear();
    for (const auto& kv : g_tune) {
        TuneEntry e;
        std::memset(&e.prob, 0, sizeof(e.prob));
        const TuneKey& k = kv.first;
        e.prob.ndim = std::get<0>(k);
        e.prob.dims[0] = std::get<1>(k);
        if (e.prob.ndim == 3) {
            e.prob.dims[1] = std::get<2>(k);
            e.prob.dims[2] = std::get<3>(k);
        } else {
            e.prob.dims[1] = std::get<3>(k);
        }
        e.prob.batch = std::get<4>(k);
        const uint32_t sb = std::get<5>(k);
        std::memcpy(&e.prob.sigma, &sb, 4);
        e.prob.T = 1;
        e.tun = kv.second;
        out->push_back(e);
    }
}

}  // namespace meta

using namespace meta;

extern "C" {

meta_status meta_tuning_set(const meta_problem* prob, const meta_tuning* tun) {
    const meta_status s = validate(prob);
    if (s != META_OK) return s;
    if (!tun) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune.erase(tune_key(prob));
        return META_OK;
    }
    const meta_status c = tuning_check(prob, tun);
    if (c != META_OK) return c;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(prob)] = *tun;
    return META_OK;
}

meta_status meta_tuning_get(const meta_problem* prob, meta_tuning* out) {
    if (!out) return META_ERR_INVALID_ARG;
    const meta_status s = validate(prob);
    if (s != META_OK) return s;
    const Layout L = make_layout(prob);
    out->ly = L.g.ly;
    out->txw = L.g.txw;
    meta_tuning tn;
    out->split = (find_tuning(prob, &tn) && tn.split > 0) ? tn.split : 1;
    if (L.ndim == 3) {
        out->lz = L.g.lz;
        out->zc_transport = L.g.zct > 0 ? L.g.zct : march_chunk(L.g, 4, 2, kTransRows);
        out->zc_advect = L.g.zca > 0 ? L.g.zca : march_chunk(L.g, 5, 2, kAdvRows);
    } else {
        out->lz = out->zc_transport = out->zc_advect = 0;
    }
    return META_OK;
}

meta_status meta_autotune(const meta_problem* prob, const float* I0, const float* J,
                          const float* p0, const float* mu, const float* rho, const float* lambda,
                          double* cost, float* grad, void* ws, size_t ws_bytes, void* stream,
                          meta_tuning* out) {
    meta_status s = adjoint_scheme(prob);
    if (s != META_OK) return s;
    meta_tuning cur;
    if (tuning_cache_lookup(prob, &cur)) {  // tuned before, in the cache file: no timing
        s = meta_tuning_set(prob, &cur);
        if (s == META_OK && out) *out = cur;
        return s;
    }
    s = meta_tuning_get(prob, &cur);
    if (s != META_OK) return s;
    const int d = prob->ndim;
    const int nz = d == 3 ? prob->dims[0] : 1, ny = prob->dims[d - 2], nx = prob->dims[d - 1];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return META_ERR_CUDA;
    }
    // one warm-up, then the median of nine timed calls
    auto time_it = [&](float* ms) -> meta_status {
        meta_status r = meta_cost_and_grad(prob, I0, J, p0, mu, rho, lambda, cost, grad, ws,
                                           ws_bytes, stream);
        if (r != META_OK) return r;
        float tk[9];
        for (int k = 0; k < 9; ++k) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return META_ERR_CUDA;
            r = meta_cost_and_grad(prob, I0, J, p0, mu, rho, lambda, cost, grad, ws, ws_bytes,
                                   stream);
            if (r != META_OK) return r;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return META_ERR_CUDA;
            if (cudaEventElapsedTime(&tk[k], e0, e1) != cudaSuccess) return META_ERR_CUDA;
        }
        std::sort(tk, tk + 9);
        *ms = tk[4];
        return META_OK;
    };
    // equal tiles of at most 32 .. 192 (one warp holds two groups of kBA outputs, so
    // multiples of 32 leave no idle half warp) that one TMA box can stage
    const int kp_s = strided_kp(prob->sigma);
    auto lens = [kp_s](int n, int q) {
        std::vector<int> v;
        for (int m : {32, 48, 64, 96, 128, 160, 192}) {
            const int l = even_tile(n, m, q);
            if (l <= kTAMax && l + kp_s <= 256 && std::find(v.begin(), v.end(), l) == v.end())
                v.push_back(l);
        }
        return v;
    };
    std::vector<std::pair<int*, std::vector<int>>> params;
    if (d == 3) {
        std::vector<int> zs;
        for (int z : {2, 4, 6, 8, 12, 16, 24, 32, 48, 64})
            if (z <= nz) zs.push_back(z);
        params.push_back({&cur.zc_transport, zs});
        params.push_back({&cur.zc_advect, zs});
        params.push_back({&cur.lz, lens(nz, kBA)});
    }
    params.push_back({&cur.ly, lens(ny, kBA)});
    {  // x-pass widths: equal tiles of at most 48 .. 256 that fit the TMA box
        std::vector<int> v;
        for (int m : {48, 64, 96, 128, 160, 192, 256}) {
            const int l = even_tile(nx, m, kBX);
            if (xpass_lw(l, xpass_r(prob->sigma), xpass_r4(prob->sigma)) <= kMaxLW &&
                std::find(v.begin(), v.end(), l) == v.end())
                v.push_back(l);
        }
        params.push_back({&cur.txw, v});
    }
    // Two sweeps of one field at a time.  Each field keeps its current value (timed
    // first) unless a candidate is at least 1 % faster, so that timing noise does
    // not move a field between values of about the same speed.
    meta_status res = META_OK;
    for (int sweep = 0; sweep < 2 && res == META_OK; ++sweep) {
        for (auto& pv : params) {
            int best_v = *pv.first;
            float best_ms = 1e30f;
            if (meta_tuning_set(prob, &cur) == META_OK) {
                res = time_it(&best_ms);
                if (res != META_OK) break;
            }
            for (int v : pv.second) {
                if (v == best_v) continue;
                const int keep = *pv.first;
                *pv.first = v;
                const bool ok = meta_tuning_set(prob, &cur) == META_OK;  // else a launch limit
                float ms = 0.f;
                if (ok) {
                    res = time_it(&ms);
                    if (res != META_OK) break;
                }
                *pv.first = keep;
                if (ok && ms < 0.99f * best_ms) {
                    best_ms = ms;
                    best_v = v;
                    *pv.first = v;
                }
            }
            *pv.first = best_v;
            if (res != META_OK) break;
        }
    }
    // batch split of the recorded plan: time plan launches
    if (res == META_OK && prob->batch > 1) {
        int best_v = cur.split, nbest = 0;
        float best_ms = 1e30f;
        for (int S : {1, 2, 4, 8, 16}) {
            if (S > prob->batch || S > kMaxSplit) break;
            cur.split = S;
            if (meta_tuning_set(prob, &cur) != META_OK) continue;
            meta_plan* pl = nullptr;
            res = meta_plan_create(prob, I0, J, p0, mu, rho, lambda, cost, grad, ws, ws_bytes, &pl);
            if (res != META_OK) break;
            float tk[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < 6 && res == META_OK; ++k) {
                if (cudaEventRecord(e0, st) != cudaSuccess ||
                    meta_plan_launch(pl, stream) != META_OK ||
                    cudaEventRecord(e1, st) != cudaSuccess ||
                    cudaEventSynchronize(e1) != cudaSuccess) {
                    res = META_ERR_CUDA;
                    break;
                }
                if (cudaEventElapsedTime(&tk[k], e0, e1) != cudaSuccess) res = META_ERR_CUDA;
            }
            std::sort(tk + 1, tk + 6);  // launch 0 warms up
            const float best = tk[3];   // median of the other five
            meta_plan_destroy(pl);
            if (res != META_OK) break;
            ++nbest;
            if (best < best_ms) {
                best_ms = best;
                best_v = S;
            }
        }
        cur.split = nbest ? best_v : cur.split;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (res != META_OK) {
        meta_tuning_set(prob, nullptr);
        return res;
    }
    res = meta_tuning_set(prob, &cur);
    if (res != META_OK) return res;
    if (out) *out = cur;
    return tuning_cache_note(prob, cur);  // merged into the cache file, if one is named
}

meta_status meta_workspace_size(const meta_problem* prob, size_t* bytes) {
    if (!bytes) return META_ERR_INVALID_ARG;
    const meta_status s = validate(prob);
    if (s != META_OK) return s;
    size_t total = make_layout(prob).total;
    const int smax = prob->batch < kMaxSplit ? prob->batch : kMaxSplit;
    for (int S = 2; S <= smax; ++S) {
        const size_t b = split_bytes(prob, S);
        total = b > total ? b : total;
    }
    *bytes = total;
    return META_OK;
}

meta_status meta_shoot_forward(const meta_problem* prob, const float* I0, const float* p0,
                               const float* mu, const float* rho, float* I1, float* p1, void* ws,
                               size_t ws_bytes, void* stream) {
    if (!I0 || !p0 || !mu || !rho) return META_ERR_INVALID_ARG;
    Ctx c;
    meta_status s = setup(prob, ws, ws_bytes, stream, &c);
    if (s != META_OK) return s;
    const Geom& g = c.L.g;
    const Coefs cf{mu, rho, nullptr, 1.f / (float)c.L.T, c.L.pdet, c.L.scheme};
    META_LAUNCH(META_K_PACK, c.st,
                launch_pack(g, c.L.ndim, I0, p0, c.states, c.states + (size_t)g.B * g.inst, c.st));
    s = run_forward(c, cf);
    if (s != META_OK) return s;
    if (I1 || p1) {
        const size_t slot = (size_t)c.L.final_slot() * 2 * g.B * g.inst;
        META_LAUNCH(META_K_UNPACK, c.st,
                    launch_unpack(g, c.L.ndim, c.states + slot,
                                  c.states + slot + (size_t)g.B * g.inst, I1, p1, c.st));
    }
    return META_OK;
}

meta_status meta_shoot_deform(const meta_problem* prob, const float* I0, const float* p0,
                              const float* mu, const float* rho, float* I1, float* p1,
                              float* phi, float* jac, void* ws, size_t ws_bytes, void* stream) {
    if (!I0 || !p0 || !mu || !rho || (!phi && !jac)) return META_ERR_INVALID_ARG;
    Ctx c;
    meta_status s = setup(prob, ws, ws_bytes, stream, &c);
    if (s != META_OK) return s;
    const Geom& g = c.L.g;
    const Coefs cf{mu, rho, nullptr, 1.f / (float)c.L.T, c.L.pdet, c.L.scheme};
    META_LAUNCH(META_K_PACK, c.st,
                launch_pack(g, c.L.ndim, I0, p0, c.states, c.states + (size_t)g.B * g.inst, c.st));
    const float* wT = nullptr;
    s = run_forward(c, cf, &wT);
    if (s != META_OK) return s;
    META_LAUNCH(META_K_DEFORM_OUT, c.st, launch_deform_out(g, c.L.ndim, wT, phi, jac, c.st));
    if (I1 || p1) {
        const size_t slot = (size_t)c.L.final_slot() * 2 * g.B * g.inst;
        META_LAUNCH(META_K_UNPACK, c.st,
                    launch_unpack(g, c.L.ndim, c.states + slot,
                                  c.states + slot + (size_t)g.B * g.inst, I1, p1, c.st));
    }
    return META_OK;
}

meta_status meta_shoot_adjoint(const meta_problem* prob, const float* mu, const float* rho,
                               const float* gI1, const float* gp1, float* gI0, float* gp0,
                               void* ws, size_t ws_bytes, void* stream) {
    if (!mu || !rho || !gI1 || !gp0) return META_ERR_INVALID_ARG;
    meta_status s = adjoint_scheme(prob);
    if (s != META_OK) return s;
    Ctx c;
    s = setup(prob, ws, ws_bytes, stream, &c);
    if (s != META_OK) return s;
    const Coefs cf{mu, rho, nullptr, 1.f / (float)c.L.T, c.L.pdet, c.L.scheme};
    // With checkpoints, an earlier adjoint left other segments in the segment
    // slots: bring the last nbuf back so that the adjoint can be called again.
    if (c.L.k) {
        const int s_last = c.L.seg_of(c.L.T - 1);
        for (int q = s_last - c.L.nbuf + 1 < 0 ? 0 : s_last - c.L.nbuf + 1;
             q <= s_last && s == META_OK; ++q)
            s = recompute_segment(c, cf, q);
        if (s != META_OK) return s;
    }
    META_LAUNCH(META_K_ADJ_INIT, c.st,
                launch_adj_init(c.L.g, c.L.ndim, cf, start_slots(c.L), c.states, c.u, gI1, gp1,
                                c.maxdisp, c.REC, c.IHP, c.PHP, c.RAW, raw_p(c), c.st));
    return run_adjoint(c, cf, 2, gp0, gI0);
}

meta_status meta_cost_and_grad(const meta_problem* prob, const float* I0, const float* J,
                               const float* p0, const float* mu, const float* rho,
                               const float* lambda, double* cost, float* grad, void* ws,
                               size_t ws_bytes, void* stream) {
    return cost_and_grad_impl(prob, I0, J, p0, mu, rho, lambda, cost, grad, ws, ws_bytes, stream,
                              nullptr);
}

struct meta_plan {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    PersistPlan* persist = nullptr;  // meta_plan_create_persistent only
};

// Records problem k on branch k % streams of one graph (fork from a root
// stream, join back); `fault` (nullable) overrides every call's fault word.
static meta_status record_branches(int n, const meta_problem* probs, const float* const* I0,
                                   const float* const* J, const float* const* p0,
                                   const float* const* mu, const float* const* rho,
                                   const float* const* lambda, double* const* cost,
                                   float* const* grad, void* const* ws, const size_t* ws_bytes,
                                   int streams, unsigned int* fault, meta_plan** plan) {
    *plan = nullptr;
    if (streams < 1) streams = 1;
    if (streams > n) streams = n;
    if (streams > 64) streams = 64;
    cudaStream_t root, br[64];
    cudaEvent_t fork, done[64];
    int made = 0;
    meta_status status = META_OK;
    cudaGraph_t graph = nullptr;
    if (cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking) != cudaSuccess) return META_ERR_CUDA;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(root);
        return META_ERR_CUDA;
    }
    for (; made < streams; ++made) {
        if (cudaStreamCreateWithFlags(&br[made], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[made], cudaEventDisableTiming) != cudaSuccess) {
            status = META_ERR_CUDA;
            break;
        }
    }
    const bool timer_was_on = g_timer.on;
    g_timer.on = false;
    if (status == META_OK &&
        cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        status = META_ERR_CUDA;
    else if (status == META_OK) {
        // fork every branch stream from the root, record problem k on branch k % streams
        if (cudaEventRecord(fork, root) != cudaSuccess) status = META_ERR_CUDA;
        for (int j = 0; j < streams && status == META_OK; ++j)
            if (cudaStreamWaitEvent(br[j], fork, 0) != cudaSuccess) status = META_ERR_CUDA;
        for (int k = 0; k < n && status == META_OK; ++k)
            status = cost_and_grad_impl(&probs[k], I0[k], J[k], p0[k], mu[k], rho[k], lambda[k],
                                        cost[k], grad[k], ws[k], ws_bytes[k], br[k % streams],
                                        fault);
        // join
        for (int j = 0; j < streams; ++j) {
            cudaEventRecord(done[j], br[j]);
            cudaStreamWaitEvent(root, done[j], 0);
        }
        const cudaError_t e = cudaStreamEndCapture(root, &graph);
        if (status == META_OK && e != cudaSuccess) status = META_ERR_CUDA;
    }
    g_timer.on = timer_was_on;
    cudaGetLastError();
    cudaGraphExec_t exec = nullptr;
    if (status == META_OK && (!graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess))
        status = META_ERR_CUDA;
    for (int j = 0; j < made; ++j) {
        cudaStreamDestroy(br[j]);
        cudaEventDestroy(done[j]);
    }
    cudaEventDestroy(fork);
    cudaStreamDestroy(root);
    if (status != META_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        return status;
    }
    meta_plan* p = new (std::nothrow) meta_plan{graph, exec};
    if (!p) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return META_ERR_INVALID_ARG;
    }
    *plan = p;
    return META_OK;
}


// The batch recorded as S sub-batches on parallel branches of one graph: the
// kernels of one branch fill the GPU while another's drain.  Sub-batch k runs
// on its own 256-byte aligned region of ws and reports faults to the first
// region's word (the header of ws); every instance is computed as in one call.
static meta_status plan_create_split(const meta_problem* prob, int S, const float* I0,
                                     const float* J, const float* p0, const float* mu,
                                     const float* rho, const float* lambda, double* cost,
                                     float* grad, void* ws, size_t ws_bytes, meta_plan** plan) {
    if (!I0 || !J || !p0 || !mu || !rho || !lambda || !cost || !ws) return META_ERR_INVALID_ARG;
    if (split_bytes(prob, S) > ws_bytes) return META_ERR_WORKSPACE;
    if ((reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return META_ERR_WORKSPACE;
    // sub-batches take the tile shapes tuned for the whole batch
    meta_tuning parent;
    if (find_tuning(prob, &parent)) {
        parent.split = 0;
        for (int k = 0; k < S; ++k) {
            int first, count;
            split_range(prob->batch, S, k, &first, &count);
            meta_problem sub = *prob;
            sub.batch = count;
            meta_tuning have;
            if (!find_tuning(&sub, &have)) meta_tuning_set(&sub, &parent);
        }
    }
    long long N = 1;
    for (int a = 0; a < prob->ndim; ++a) N *= prob->dims[a];
    std::vector<meta_problem> probs(S);
    std::vector<const float*> vI0(S), vJ(S), vp0(S), vmu(S), vrho(S), vlam(S);
    std::vector<double*> vcost(S);
    std::vector<float*> vgrad(S);
    std::vector<void*> vws(S);
    std::vector<size_t> vwsb(S);
    size_t off = 0;
    for (int k = 0; k < S; ++k) {
        int first, count;
        split_range(prob->batch, S, k, &first, &count);
        probs[k] = *prob;
        probs[k].batch = count;
        vI0[k] = I0 + first * N;
        vJ[k] = J + first * N;
        vp0[k] = p0 + first * N;
        vmu[k] = mu + first;
        vrho[k] = rho + first;
        vlam[k] = lambda + first;
        vcost[k] = cost + 3 * (long long)first;
        vgrad[k] = grad ? grad + first * N : nullptr;
        const size_t b = align_up(make_layout(&probs[k]).total, kAlign);
        vws[k] = static_cast<char*>(ws) + off;
        vwsb[k] = b;
        off += b;
    }
    return record_branches(S, probs.data(), vI0.data(), vJ.data(), vp0.data(), vmu.data(),
                           vrho.data(), vlam.data(), vcost.data(), vgrad.data(), vws.data(),
                           vwsb.data(), S, reinterpret_cast<unsigned int*>(ws), plan);
}

meta_status meta_plan_create(const meta_problem* prob, const float* I0, const float* J,
                             const float* p0, const float* mu, const float* rho,
                             const float* lambda, double* cost, float* grad, void* ws,
                             size_t ws_bytes, meta_plan** plan) {
    if (!plan) return META_ERR_INVALID_ARG;
    *plan = nullptr;
    size_t need = 0;
    meta_status s = meta_workspace_size(prob, &need);
    if (s != META_OK) return s;
    s = adjoint_scheme(prob);
    if (s != META_OK) return s;
    meta_tuning tn;
    const int S = (find_tuning(prob, &tn) && tn.split > 1 && tn.split <= prob->batch) ? tn.split : 1;
    if (S > 1) return plan_create_split(prob, S, I0, J, p0, mu, rho, lambda, cost, grad, ws,
                                        ws_bytes, plan);
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return META_ERR_CUDA;
    const bool timer_was_on = g_timer.on;
    g_timer.on = false;  // the recorded sequence carries no timing events
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        g_timer.on = timer_was_on;
        cudaStreamDestroy(cs);
        return META_ERR_CUDA;
    }
    s = meta_cost_and_grad(prob, I0, J, p0, mu, rho, lambda, cost, grad, ws, ws_bytes, cs);
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    g_timer.on = timer_was_on;
    cudaStreamDestroy(cs);
    if (s != META_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return s != META_OK ? s : META_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return META_ERR_CUDA;
    }
    meta_plan* p = new (std::nothrow) meta_plan{graph, exec};
    if (!p) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return META_ERR_INVALID_ARG;
    }
    *plan = p;
    return META_OK;
}

meta_status meta_plan_create_group(int n, const meta_problem* probs, const float* const* I0,
                                   const float* const* J, const float* const* p0,
                                   const float* const* mu, const float* const* rho,
                                   const float* const* lambda, double* const* cost,
                                   float* const* grad, void* const* ws, const size_t* ws_bytes,
                                   int streams, meta_plan** plan) {
    if (!plan || n < 1 || !probs || !I0 || !J || !p0 || !mu || !rho || !lambda || !cost ||
        !grad || !ws || !ws_bytes)
        return META_ERR_INVALID_ARG;
    *plan = nullptr;
    for (int k = 0; k < n; ++k) {
        size_t need = 0;
        meta_status s = meta_workspace_size(&probs[k], &need);
        if (s == META_OK) s = adjoint_scheme(&probs[k]);
        if (s != META_OK) return s;
        if (ws_bytes[k] < need) return META_ERR_WORKSPACE;
    }
    return record_branches(n, probs, I0, J, p0, mu, rho, lambda, cost, grad, ws, ws_bytes,
                           streams, nullptr, plan);
}

meta_status meta_plan_create_persistent(int n, const meta_problem* probs,
                                        const float* const* I0, const float* const* J,
                                        const float* const* p0, const float* const* mu,
                                        const float* const* rho, const float* const* lambda,
                                        double* const* cost, float* const* grad, void* const* ws,
                                        const size_t* ws_bytes, meta_plan** plan) {
    if (!plan) return META_ERR_INVALID_ARG;
    *plan = nullptr;
    if (n < 1 || !probs || !I0 || !J || !p0 || !mu || !rho || !lambda || !cost || !grad || !ws ||
        !ws_bytes)
        return META_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k) {
        size_t need = 0;
        meta_status s = meta_workspace_size(&probs[k], &need);
        if (s == META_OK) s = adjoint_scheme(&probs[k]);
        if (s != META_OK) return s;
        if (probs[k].scheme != META_SCHEME_SL || probs[k].p_update != META_P_UPDATE_DIV)
            return META_ERR_UNSUPPORTED;
        if (ws_bytes[k] < need) return META_ERR_WORKSPACE;
        if (!grad[k]) return META_ERR_INVALID_ARG;
    }
    // each problem's launch sequence, recorded (nothing is launched)
    std::vector<std::vector<PRec>> recs(n);
    const bool timer_was_on = g_timer.on;
    g_timer.on = false;
    meta_status status = META_OK;
    for (int k = 0; k < n && status == META_OK; ++k) {
        recorder() = &recs[k];
        status = cost_and_grad_impl(&probs[k], I0[k], J[k], p0[k], mu[k], rho[k], lambda[k],
                                    cost[k], grad[k], ws[k], ws_bytes[k], nullptr, nullptr);
        recorder() = nullptr;
        // every phase reports a dependency timeout to its problem's status word
        for (PRec& e : recs[k]) e.a.fault = static_cast<unsigned int*>(ws[k]);
    }
    g_timer.on = timer_was_on;
    if (status != META_OK) return status;
    PersistPlan* pp = nullptr;
    {
        const cudaError_t e = persist_build(recs, &pp);
        if (e == cudaErrorNotSupported) return META_ERR_UNSUPPORTED;
        if (e != cudaSuccess) return META_ERR_CUDA;
    }
    // one graph: clear the counters, then the persistent kernel
    cudaStream_t st = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) status = META_ERR_CUDA;
    if (status == META_OK &&
        cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        status = META_ERR_CUDA;
    else if (status == META_OK) {
        const cudaError_t e = persist_launch(pp, st, 5000000000ull, -1);
        const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) status = META_ERR_CUDA;
    }
    cudaGetLastError();
    if (status == META_OK && (!graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess))
        status = META_ERR_CUDA;
    if (st) cudaStreamDestroy(st);
    meta_plan* p = status == META_OK ? new (std::nothrow) meta_plan{graph, exec} : nullptr;
    if (!p) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        persist_free(pp);
        return status == META_OK ? META_ERR_INVALID_ARG : status;
    }
    p->persist = pp;
    *plan = p;
    return META_OK;
}

meta_status meta_plan_status(meta_plan* plan, int clear, void* stream, unsigned int* bits) {
    if (!plan || !bits) return META_ERR_INVALID_ARG;
    *bits = 0u;
    if (!plan->persist) return META_OK;
    if (persist_status(plan->persist, clear, static_cast<cudaStream_t>(stream), bits) !=
        cudaSuccess)
        return META_ERR_CUDA;
    return (*bits & 1u) ? META_ERR_TIMEOUT : META_OK;
}

meta_status meta_plan_selftest_timeout(meta_plan* plan, int hold, unsigned long long limit_ns,
                                       void* stream) {
    if (!plan || !plan->persist) return META_ERR_INVALID_ARG;
    if (hold < 0 || hold >= persist_problems(plan->persist)) return META_ERR_INVALID_ARG;
    if (limit_ns < 1000000ull || limit_ns > 2000000000ull) return META_ERR_INVALID_ARG;
    return map_status(persist_launch(plan->persist, static_cast<cudaStream_t>(stream), limit_ns,
                                     hold));
}

meta_status meta_plan_launch(meta_plan* plan, void* stream) {
    if (!plan) return META_ERR_INVALID_ARG;
    return map_status(cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)));
}

meta_status meta_plan_destroy(meta_plan* plan) {
    if (!plan) return META_OK;
    cudaGraphExecDestroy(plan->exec);
    cudaGraphDestroy(plan->graph);
    persist_free(plan->persist);
    delete plan;
    return META_OK;
}

meta_status meta_selftest_timeout(void* ws, size_t ws_bytes, unsigned long long limit_ns,
                                  void* stream) {
    if (!ws || ws_bytes < 16 || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
        return META_ERR_WORKSPACE;
    if (limit_ns < 1000000ull || limit_ns > 2000000000ull) return META_ERR_INVALID_ARG;
    return map_status(launch_wait_selftest(static_cast<unsigned int*>(ws), limit_ns,
                                           static_cast<cudaStream_t>(stream)));
}

meta_status meta_workspace_status(void* ws, size_t ws_bytes, int clear, void* stream,
                                  unsigned int* fault_bits) {
    if (!ws || ws_bytes < 16 || !fault_bits) return META_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int* f = static_cast<unsigned int*>(ws);  // off_fault == 0
    if (cudaStreamSynchronize(st) != cudaSuccess) return META_ERR_CUDA;
    if (cudaMemcpy(fault_bits, f, sizeof(unsigned int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return META_ERR_CUDA;
    if (clear) {
        if (cudaMemsetAsync(f, 0, sizeof(unsigned int), st) != cudaSuccess) return META_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return META_ERR_CUDA;
    }
    return (*fault_bits & kFaultTmaTimeout) ? META_ERR_TIMEOUT : META_OK;
}

meta_status meta_timer_start(int cap) {
    if (cap < 1 || cap > (1 << 22)) return META_ERR_INVALID_ARG;
    Timer& T = g_timer;
    if ((int)T.ev.size() < 2 * cap) {
        const size_t old = T.ev.size();
        T.ev.resize(2 * (size_t)cap);
        for (size_t i = old; i < T.ev.size(); ++i)
            if (cudaEventCreate(&T.ev[i]) != cudaSuccess) {
                T.ev.resize(i);
                return META_ERR_CUDA;
            }
    }
    T.cls.assign(cap, -1);
    T.cap = cap;
    T.used = 0;
    T.on = true;
    return META_OK;
}

meta_status meta_timer_stop(float* ms_per_class, int* launches_per_class) {
    Timer& T = g_timer;
    if (!T.on) return META_ERR_INVALID_ARG;
    T.on = false;
    for (int k = 0; k < META_K_COUNT; ++k) {
        if (ms_per_class) ms_per_class[k] = 0.f;
        if (launches_per_class) launches_per_class[k] = 0;
    }
    for (int i = 0; i < T.used; ++i) {
        if (cudaEventSynchronize(T.ev[2 * i + 1]) != cudaSuccess) return META_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, T.ev[2 * i], T.ev[2 * i + 1]) != cudaSuccess)
            return META_ERR_CUDA;
        const int k = T.cls[i];
        if (k >= 0 && k < META_K_COUNT) {
            if (ms_per_class) ms_per_class[k] += ms;
            if (launches_per_class) launches_per_class[k] += 1;
        }
    }
    T.used = 0;
    return META_OK;
}

const char* meta_kernel_name(int k) {
    static const char* names[META_K_COUNT] = {
        "pack", "xpass_m", "strided_fwd", "advect", "cost", "adj_init",
        "adj_pre", "adj_gather", "xpass_adj", "strided_adj", "adj_gradp", "unpack",
        "deform", "deform_out", "adj_jac", "euler"};
    return (k >= 0 && k < META_K_COUNT) ? names[k] : "unknown";
}

const char* meta_status_string(meta_status s) {
    switch (s) {
        case META_OK: return "ok";
        case META_ERR_INVALID_ARG: return "invalid argument";
        case META_ERR_SHAPE: return "unsupported shape";
        case META_ERR_WORKSPACE: return "workspace too small or misaligned";
        case META_ERR_CUDA: return "CUDA error";
        case META_ERR_TIMEOUT: return "device-side wait timed out";
        case META_ERR_NONFINITE: return "non-finite value";
        case META_ERR_UNSUPPORTED: return "unsupported device or driver";
        case META_ERR_FORMAT: return "malformed or mismatched saved state";
        case META_ERR_IO: return "file I/O error";
    }
    return "unknown status";
}

meta_status meta_trace_set(meta_trace_fn fn, void* user) {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    g_trace_fn = fn;
    g_trace_user = fn ? user : nullptr;
    return META_OK;
}

meta_status meta_trace_selftest(void) {
    Range outer("meta.selftest");
    {
        Range inner("meta.selftest.inner");
    }
    return META_OK;
}

}  // extern "C"
