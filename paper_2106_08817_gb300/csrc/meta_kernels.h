// meta_kernels.h -- internal launchers of the sm_103a kernels (not part of the C ABI).
#pragma once

#include "meta_common.cuh"
#include "meta.h"

#include <vector>

namespace meta {

// ---------------------------------------------------------------- recording
// Launches of one call, recorded instead of launched (meta_persist.cu replays
// them as phases of one persistent kernel).  While recorder() points to a
// vector, each launcher below of the semi-Lagrangian path appends one record
// per kernel launch (and run_forward one per memset) and launches nothing.
enum PKind {
    PK_ZERO = 0,   // zero n 32-bit words at md
    PK_PACK,       // k_pack
    PK_XPASS,      // k_xpass (sub: GRADP)
    PK_STRIDED,    // k_strided (sub: AXIS)
    PK_ADVECT,     // k_advect2d / 3d (sub: PDET)
    PK_COSTP,      // k_cost_partials
    PK_ADJINIT,    // k_adj_init (sub: FROM_J)
    PK_COSTF,      // k_cost_final
    PK_ADJREC,     // k_adj_records
    PK_TRANS,      // k_adj_transport2d / 3d
    PK_GRADP,      // k_adj_gradp2d / k_adj_gradp (sub: PDET)
    PK_COUNT
};

// Every argument any recorded kernel takes; each kind reads its own fields.
struct PArgs {
    Geom g;
    Coefs cf;
    Slots sl;
    int t, mode, zc, i0, i1, i2, n;
    float f0;
    const float* c[4];
    float* w[7];
    double* d[2];
    unsigned int* md;     // max displacement per step (written by the advect)
    const unsigned int* cmd;  // the same, read
    unsigned int* fault;  // workspace status word
};

struct PRec {
    int kind, ndim, sub, kc;  // kc: tap chunks of 8 (taps.kp / 8)
    dim3 grid;
    int bx, by;               // threads of the recorded block (x, y)
    size_t smem;              // shared memory the body needs
    PArgs a;
    int ntm;                  // tensor maps used (by value)
    CUtensorMap tm[3];
    int has_taps;
    Taps taps;
};

std::vector<PRec>*& recorder();

// The persistent kernel's plan (meta_persist.cu): the recorded launches of
// every problem as device tables, and the control block of one launch.
struct PersistPlan;
cudaError_t persist_build(const std::vector<std::vector<PRec>>& recs, PersistPlan** out);
// Clears the counters and launches the kernel on st; dependency waits give up
// after limit_ns; hold >= 0 withholds the completion of that problem's first
// phase (self-test of the bounded waits).
cudaError_t persist_launch(PersistPlan* p, cudaStream_t st, unsigned long long limit_ns, int hold);
cudaError_t persist_status(PersistPlan* p, int clear, cudaStream_t st, unsigned* bits);
void persist_free(PersistPlan* p);
int persist_problems(const PersistPlan* p);
long long persist_tiles(const PersistPlan* p);
int persist_grid(const PersistPlan* p);

// Blur passes (meta_blur.cu).
size_t xpass_smem(int ndim, bool gradp, int txw, int r, int r4);
size_t strided_smem(int len, int kp);

// Failure-path self-test: a bounded mbarrier wait that runs out after limit_ns
// and latches the timeout bit in *fault.
cudaError_t launch_wait_selftest(unsigned int* fault, unsigned long long limit_ns, cudaStream_t st);

// x-pass.  gradp: reads I slice (sliceI + b) with a one-voxel y/z halo and p
// slice (sliceP + b) through tmI / tmP, writes NDIM component slices
// out_slice0 + a*B + b.  Plain: reads slice sliceI + s through tmI and writes
// out_slice0 + s, for s < nslices.
cudaError_t launch_xpass(int ndim, bool gradp, const CUtensorMap& tmI, const CUtensorMap& tmP,
                         const Taps& taps, const Geom& g, int sliceI, int sliceP, const float* pin, int out_slice0,
                         int nslices, float* out, unsigned int* fault, cudaStream_t st);

// Strided pass along `axis` (2-D: 0 = y; 3-D: 1 = y, 0 = z) of slices
// in_slice0 + s -> out_slice0 + s, s < nslices, multiplied by
// scale_mul * scale[s % B] when scale is not null.
cudaError_t launch_strided(int ndim, int axis, const CUtensorMap& tm, const Taps& taps,
                           const Geom& g, int in_slice0, int out_slice0, int nslices,
                           const float* scale, float scale_mul, float* out, unsigned int* fault,
                           cudaStream_t st);

// Pointwise / gather kernels (meta_step.cu).  Buffers are pitched slices of
// g.inst floats; `states` holds slice (t*2 + f)*B + b for f = 0 (I), 1 (p);
// `u` holds slice (t*NDIM + a)*B + b.
cudaError_t launch_pack(const Geom& g, int ndim, const float* I0, const float* p0, float* dstI,
                        float* dstP, cudaStream_t st);
cudaError_t launch_unpack(const Geom& g, int ndim, const float* srcI, const float* srcP,
                          float* I1, float* p1, cudaStream_t st);
// Forward step t: reads state slot sl.st and u slot sl.ut, writes slot sl.st1.
cudaError_t launch_advect(const Geom& g, int ndim, const Coefs& c, int t, const Slots& sl,
                          float* states, const float* u, unsigned int* maxdisp,
                          const CUtensorMap* maps, unsigned int* fault, cudaStream_t st);
// Eulerian (hybrid = false) or hybrid step t: state slot sl.st -> sl.st1
// with u slot sl.ut; the hybrid also records max |d| of step t in maxdisp.
cudaError_t launch_euler(const Geom& g, int ndim, const Coefs& c, int t, const Slots& sl,
                         bool hybrid, float* states, const float* u, unsigned int* maxdisp,
                         cudaStream_t st);
// Deformation step t: w_{t+1} = (y - x) + S(y) w_t from u slot su, with
// w = phi - Id in slices a*B + b of win / wout (win NULL: w_t = 0).
cudaError_t launch_deform(const Geom& g, int ndim, const Coefs& c, int su, const float* u,
                          const float* win, float* wout, cudaStream_t st);
// phi - Id (contiguous [B][ndim][N]) and det D phi ([B][N]) from pitched w;
// either output may be NULL.
cudaError_t launch_deform_out(const Geom& g, int ndim, const float* w, float* phi, float* jac,
                              cudaStream_t st);
// Adjoint (meta_adjoint.cu).  `rec` holds the records of one adjoint step:
// slice (k * B + b), k = 0 foot cell (int bits), 1..NDIM f per axis, NDIM+1
// I^', NDIM+2 p~^, NDIM+3 div^.  Ihp / php: the S^T accumulators.
// Eq. 4 partial sums (states sl.sT, sl.s0, u sl.u0), their reduction into
// cost[B][3], and the adjoint start from I^_T = I_T - J, p^_T = 0 (k_adj_init:
// the records of step T-1, state sl.st1, u sl.ut1, and for the Eulerian and
// hybrid schemes the raw adjoints in rawI / rawP).
cudaError_t launch_cost(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                        const float* states, const float* u, const float* J,
                        const unsigned int* maxdisp, float* rec, float* Ihp, float* php,
                        float* rawI, float* rawP, double* partials, int nblk, double* cost,
                        cudaStream_t st);
// Records of step T-1 from given gradients gI1, gp1 (gp1 nullable: zero).
cudaError_t launch_adj_init(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                            const float* states, const float* u, const float* gI1,
                            const float* gp1, const unsigned int* maxdisp, float* rec, float* Ihp,
                            float* php, float* rawI, float* rawP, cudaStream_t st);
// Eulerian / hybrid schemes (c.scheme 1 / 2): the start above also writes the raw
// adjoints of (I_T, p_T) into rawI / rawP (Eulerian) or rawP (hybrid, whose
// records are those of its semi-Lagrangian image step).  One Eulerian adjoint
// step up to v^ (Ihp, php, vh from rawI, rawP, state sl.st, u sl.ut), and the
// hybrid's Eulerian momentum part added after the transport.
cudaError_t launch_euler_adj(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                             const float* states, const float* u, const float* rawI,
                             const float* rawP, float* Ihp, float* php, float* vh,
                             cudaStream_t st);
cudaError_t launch_hybrid_p(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                            const float* states, const float* u, const float* rawP, float* php,
                            float* vh, cudaStream_t st);
// Records of a step (state sl.st1, u sl.ut1) from pitched raw adjoints.
cudaError_t launch_adj_records(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                               const float* states, const float* u, const float* rawI,
                               const float* rawP, float* rec, cudaStream_t st);
// S^T of I^' and p~^ into Ihp / php and v^ (d slices) into vh, for step t
// (state slot sl.st).
// In 3-D, maps[0..2] are the transport's tensor maps (records 0..5, div^, and
// the states), see encode_map5.
cudaError_t launch_adj_transport(const Geom& g, int ndim, const Coefs& c, int t, const Slots& sl,
                                 const CUtensorMap* maps, const float* states,
                                 const unsigned int* maxdisp,
                                 const float* rec, float* vh, float* Ihp, float* php,
                                 unsigned int* fault, cudaStream_t st);
// I^_t, p^_t from Ihp / php and m^ (state slot sl.st), then by mode: 0 the
// records of step t-1 (state sl.st1, u sl.ut1); 3 raw I^_t, p^_t into rawI /
// rawP; at t = 0, 1 the cost gradient (u sl.u0) and 2 the shooting adjoint,
// into contiguous grad_or_gp0 / gI0 (gI0 nullable).
// Det momentum update (c.pdet): adds sum_e D_e^T (div^ (cof(M) - Id)_ae) to
// v^_a (d slices of vh), M = Id - dt Dv_t from u slot sl.ut, div^ from rec.
cudaError_t launch_adj_jacT(const Geom& g, int ndim, const Coefs& c, const Slots& sl,
                            const float* u, const float* rec, float* vh, cudaStream_t st);
cudaError_t launch_adj_gradp(const Geom& g, int ndim, const Coefs& c, int t, int mode,
                             const Slots& sl, const float* states, const float* u,
                             const unsigned int* maxdisp, const float* mh, float* Ihp, float* php,
                             float* rec, float* rawI, float* rawP, float* grad_or_gp0,
                             float* gI0, cudaStream_t st);

// The process-wide tile-shape table (meta_api.cu) as seen by the on-disk
// cache (meta_tuning.cu).
struct TuneEntry {
    meta_problem prob;  // ndim, dims, batch, sigma (the key); T = 1, the rest 0
    meta_tuning tun;
};
meta_status tuning_check(const meta_problem* prob, const meta_tuning* tun);
void tuning_snapshot(std::vector<TuneEntry>* out);
// meta_autotune's use of the cache file named by meta_tuning_cache: a hit
// (an entry for this shape read from the file) skips the timing; a new result
// is merged into the file.
bool tuning_cache_lookup(const meta_problem* prob, meta_tuning* tun);
meta_status tuning_cache_note(const meta_problem* prob, const meta_tuning& tun);

}  // namespace meta
