/*
 * meta.h -- C ABI of the GB300 (sm_103a) library for semi-Lagrangian geodesic
 * shooting in Metamorphosis / LDDMM image registration and for the gradient of
 * the inexact-matching cost with respect to the initial momentum.
 *
 * Method: A. François, P. Gori, J. Glaunès, "Metamorphic image registration
 * using a semi-Lagrangian scheme", arXiv:2106.08817.
 *
 * What one shooting step computes (Eq. 3, integrated in the semi-Lagrangian
 * form of Sec. 2.3, Eq. 5-9), with dt = 1/T, voxel units, axis 0 first:
 *
 *     v   = -rho * K_sigma * (p grad I)        Gaussian RKHS kernel K (Sec. 2.1)
 *     y   = x - dt v                          backtracked grid, clamped to the domain
 *     I~  = I(y), p~ = p(y)                   bi/trilinear interpolation
 *     p'  = p~ (1 - dt div v)                 continuity equation (Eq. 7-9)
 *     I'  = I~ + dt mu p~                     image evolution (Eq. 1 / Eq. 5)
 *
 * rho plays the role of rho/mu in Eq. 3, so mu = 0, rho = 1 is LDDMM (Sec. 2.1).
 * Cost (Eq. 4), per instance, returned as three terms:
 *
 *     L = 1/2 sum (I_T - J)^2 + lambda [ <m0, K m0> + rho sum p0^2 ],  m0 = p0 grad I_0
 *
 * Discrete conventions: K has taps exp(-k^2 / (2 sigma^2)), |k| <= ceil(3 sigma),
 * normalised to sum 1, applied separably with zero padding outside the domain;
 * grad and div use central differences with the edge neighbour replicated;
 * interpolation clamps the foot to [0, n-1] per axis.  The gradient is the
 * exact transpose of this discrete scheme (what automatic differentiation of
 * the scheme gives, Sec. 3), computed by a hand-written adjoint.
 *
 * Conventions of every call:
 *   - Arrays are FP32, C-contiguous [batch, (D,) H, W] (axis 0 first), device
 *     pointers owned by the caller.  mu, rho, lambda are device arrays [batch].
 *   - `ws` is a device workspace of at least meta_workspace_size() bytes, owned
 *     by the caller, 256-byte aligned.  The library allocates nothing.  Its
 *     first 16 bytes hold the device fault word: zero them once before the
 *     first call (e.g. cudaMemset of the whole workspace).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     only enqueues work on it (no host synchronisation, no host<->device
 *     copies); outputs are valid once the stream has reached them.
 *   - Errors are returned as codes; nothing aborts.  Faults detected on the
 *     device (a bounded wait that ran out) are latched in the workspace and
 *     returned by meta_workspace_status().
 *   - Calls that share a workspace must be ordered on one stream.
 */
#ifndef META_H
#define META_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    META_OK = 0,
    META_ERR_INVALID_ARG = 1, /* null pointer, bad T / sigma / batch / ndim */
    META_ERR_SHAPE = 2,       /* an extent < 2, or a size beyond the limits below */
    META_ERR_WORKSPACE = 3,   /* ws too small or misaligned */
    META_ERR_CUDA = 4,        /* a CUDA runtime or driver call failed */
    META_ERR_TIMEOUT = 5,     /* a device-side bounded wait ran out */
    META_ERR_NONFINITE = 6,   /* reserved: non-finite cost detected */
    META_ERR_UNSUPPORTED = 7, /* no sm_103a device, or the driver lacks TMA support */
    META_ERR_FORMAT = 8,      /* a saved optimiser state or tuning cache is malformed, or
                                 does not match the problem (shape, m, version, checksum) */
    META_ERR_IO = 9           /* a file could not be opened, read, written or renamed */
} meta_status;

/* Shape of one batch of independent registration problems. */
typedef struct {
    int ndim;     /* 2 or 3 */
    int dims[3];  /* extents, axis 0 first: (H, W) or (D, H, W); each in [2, 65536] */
    int batch;    /* number of independent instances, >= 1 */
    int T;        /* number of time steps, dt = 1/T, in [1, 4096] */
    float sigma;  /* std (voxels) of the Gaussian RKHS kernel, in (0, 18] */
    int ckpt_stride; /* 0 or 1: keep every state (fastest); k in [2, T-1]: keep every
                        k-th state plus the states of two segments of k steps (one
                        where two would not be smaller than the whole trajectory),
                        and recompute every other segment from its checkpoint during
                        the adjoint (step checkpointing), trading k forward steps of
                        compute per segment for memory */
    int p_update;    /* momentum update of a step: META_P_UPDATE_DIV (0, the default),
                        p' = p~ (1 - dt div v), the first-order Jacobian of the backtrack
                        (Eq. 9); or META_P_UPDATE_DET (1), p' = p~ det(Id - dt Dv), its
                        exact Jacobian, Dv_ae = D_e v_a by central differences.  Every
                        call on one trajectory must use the same value. */
    int scheme;      /* integration scheme (Sec. 2.3): META_SCHEME_SL (0, the method:
                        semi-Lagrangian I and p); META_SCHEME_EULER (1: explicit Euler
                        steps of Eq. 5, I' = I - dt <grad I, v> + dt mu p, and of the
                        conservative Eq. 7, p' = p - dt div(p v), central differences);
                        META_SCHEME_HYBRID (2: the semi-Lagrangian I' with that Eulerian
                        p').  Every call takes every scheme; the adjoint is the exact
                        transpose of the chosen one.  META_P_UPDATE_DET requires
                        META_SCHEME_SL. */
} meta_problem;

#define META_P_UPDATE_DIV 0
#define META_P_UPDATE_DET 1
#define META_SCHEME_SL 0
#define META_SCHEME_EULER 1
#define META_SCHEME_HYBRID 2

/* Bytes of workspace that every call below needs for this problem (enough
 * for any batch split of meta_plan_create as well).
 * With ckpt_stride <= 1 the workspace holds the whole trajectory (I_t, p_t),
 * t = 0..T, and the smoothed momenta u_t = K(p_t grad I_t), t < T, so that the
 * adjoint needs no recomputation: about (2(T+1) + d T + 4d + 6) * batch *
 * voxels * 4 bytes.  With ckpt_stride = k > 1: about
 * (2(ceil(T/k) + k) + d(k+1) + 4d + 8) * batch * voxels * 4 bytes. */
meta_status meta_workspace_size(const meta_problem* prob, size_t* bytes);

/* Forward shooting (Eq. 3, Sec. 2.3): (I0, p0) -> (I1, p1) = (I_T, p_T).
 * I1, p1 may be NULL (the trajectory is still kept in ws for
 * meta_shoot_adjoint).  mu and rho: device [batch]. */
meta_status meta_shoot_forward(const meta_problem* prob, const float* I0, const float* p0,
                               const float* mu, const float* rho, float* I1, float* p1,
                               void* ws, size_t ws_bytes, void* stream);

/* Forward shooting that also integrates the deformation of the grid (the
 * deformation grids of Fig. 1-2, built from all the v_t of the shot):
 *
 *     phi_0 = Id,   phi_{t+1} = phi_t o (Id - dt v_t),
 *
 * composed at the same clamped feet y = x - dt v_t as the image, by the same
 * bi/trilinear interpolation: phi_{t+1}(x) = S(y) phi_t.  For mu = 0 this is the
 * map the image is carried by: an image affine in x is transported exactly as
 * I_T = I_0 o phi_T.
 *   phi: device float [batch][ndim][(D,) H, W], component a = phi_T(x)_a - x_a
 *        (axis 0 first), in voxels; may be NULL.
 *   jac: device float [batch, (D,) H, W] = det D phi_T, with D the central
 *        difference inside the domain and the one-sided difference on its two
 *        edge layers per axis (so det D Id = 1 everywhere); may be NULL.
 * At least one of phi, jac is not NULL (else META_ERR_INVALID_ARG).  I1, p1 as
 * in meta_shoot_forward, and the trajectory is left in ws for
 * meta_shoot_adjoint in the same way.  Same workspace as every other call. */
meta_status meta_shoot_deform(const meta_problem* prob, const float* I0, const float* p0,
                              const float* mu, const float* rho, float* I1, float* p1,
                              float* phi, float* jac, void* ws, size_t ws_bytes, void* stream);

/* Adjoint of the shooting map, run on the trajectory that the last
 * meta_shoot_forward left in ws (same prob, mu, rho).  Given gI1, gp1, the
 * gradient of a scalar with respect to I_T and p_T (gp1 may be NULL: zero),
 * writes its gradient with respect to p0 (gp0) and, if gI0 is not NULL, I0.
 * This is the discrete transpose of every step, run from t = T-1 down to 0.
 * With ckpt_stride > 1 it first recomputes the segments that the forward left in
 * place (the last one or two) from their checkpoints, so it may be called again on
 * the same trajectory. */
meta_status meta_shoot_adjoint(const meta_problem* prob, const float* mu, const float* rho,
                               const float* gI1, const float* gp1, float* gI0, float* gp0,
                               void* ws, size_t ws_bytes, void* stream);

/* Cost of Eq. 4 and its gradient with respect to p0, per instance.
 * cost: device double [batch][3] = { 1/2 sum (I_T - J)^2,
 *                                    lambda <m0, K m0>,
 *                                    lambda rho sum p0^2 }.
 * grad: device float [batch, (D,) H, W] = dL/dp0 (may be NULL: cost only).
 * Summation of the cost is deterministic (fixed tree, FP64 partials). */
meta_status meta_cost_and_grad(const meta_problem* prob, const float* I0, const float* J,
                               const float* p0, const float* mu, const float* rho,
                               const float* lambda, double* cost, float* grad, void* ws,
                               size_t ws_bytes, void* stream);

/* A recorded meta_cost_and_grad call.  meta_plan_create records the whole
 * launch sequence of one call, for exactly these arguments, into a CUDA graph
 * (on a private stream; nothing runs yet).  meta_plan_launch replays it on
 * `stream` with a single graph launch: the caller updates the contents of I0,
 * J, p0, mu, rho, lambda in place between launches (e.g. one gradient-descent
 * step on p0) and reads cost and grad after the stream reaches them.  The plan
 * keeps the pointers, not the data; the buffers and ws must outlive it, and
 * launches that share ws must be ordered on one stream.  Same status codes as
 * meta_cost_and_grad; creation may allocate driver resources for the graph. */
typedef struct meta_plan meta_plan;
meta_status meta_plan_create(const meta_problem* prob, const float* I0, const float* J,
                             const float* p0, const float* mu, const float* rho,
                             const float* lambda, double* cost, float* grad, void* ws,
                             size_t ws_bytes, meta_plan** plan);
/* The same for n independent problems of different shapes, sizes, T or sigma
 * (2-D and 3-D may be mixed).  Problem k has its own inputs, outputs and
 * workspace (arrays of n host-side entries, each a device pointer as in
 * meta_cost_and_grad).  The n calls are recorded into one CUDA graph as
 * parallel branches (up to `streams` concurrent ones), so a single
 * meta_plan_launch runs the whole mixed batch and independent problems
 * overlap on the GPU. */
meta_status meta_plan_create_group(int n, const meta_problem* probs, const float* const* I0,
                                   const float* const* J, const float* const* p0,
                                   const float* const* mu, const float* const* rho,
                                   const float* const* lambda, double* const* cost,
                                   float* const* grad, void* const* ws, const size_t* ws_bytes,
                                   int streams, meta_plan** plan);
/* The same n problems (arguments as meta_plan_create_group) in ONE persistent
 * kernel launch: many registrations of uneven sizes, 2-D and 3-D, T and sigma
 * (each one cost_and_grad: Eq. 3 shooting in the semi-Lagrangian form of
 * Sec. 2.3, the Eq. 4 cost and its adjoint).  Every problem's launch sequence
 * is recorded once into per-problem phases (one per kernel launch of its call,
 * each with that launch's tiles); the phases of all problems are interleaved
 * by progress into one order, and the kernel's CTAs take tiles from one work
 * counter in that order.  A tile waits (bounded spin) until its problem's
 * earlier phases are complete, then runs the same kernel body on that tile, so
 * every problem's cost and grad are bit-identical to its own
 * meta_cost_and_grad.  Supported: the semi-Lagrangian scheme with the default
 * momentum update (else META_ERR_UNSUPPORTED), any checkpoint stride; x tiles
 * of at most 128 voxels (tuned wider ones give META_ERR_UNSUPPORTED).  Creation
 * allocates the plan's device tables (phases, tensor maps, taps, counters) and
 * records one CUDA graph: the counters cleared, then the kernel.  Each
 * workspace's header must be zero as for meta_cost_and_grad. */
meta_status meta_plan_create_persistent(int n, const meta_problem* probs,
                                        const float* const* I0, const float* const* J,
                                        const float* const* p0, const float* const* mu,
                                        const float* const* rho, const float* const* lambda,
                                        double* const* cost, float* const* grad, void* const* ws,
                                        const size_t* ws_bytes, meta_plan** plan);
meta_status meta_plan_launch(meta_plan* plan, void* stream);
/* Status of a plan's launches since the status was last cleared.  Persistent
 * plans: bit 0 = a dependency wait ran out (after 5 s) and that launch
 * was abandoned (its results are invalid; returns META_ERR_TIMEOUT); the
 * waiting problem's workspace status word has bit 0 as well.  Other plans
 * report their status through their workspaces (meta_workspace_status) and give
 * 0 here.  Synchronises `stream`; clear != 0 resets the word. */
meta_status meta_plan_status(meta_plan* plan, int clear, void* stream, unsigned int* bits);
/* Self-test of the persistent kernel's failure detection: one launch in which
 * the first phase of problem `hold` never reports its tiles as complete and
 * dependency waits give up after limit_ns (in [1 ms, 2 s]).  The problem's
 * second phase waits until the limit runs out, the launch is abandoned, and
 * meta_plan_status reports META_ERR_TIMEOUT; nothing faults.  After clearing
 * the plan's status and the workspaces' status words, meta_plan_launch runs
 * normally.  META_ERR_INVALID_ARG for a plan that is not persistent. */
meta_status meta_plan_selftest_timeout(meta_plan* plan, int hold, unsigned long long limit_ns,
                                       void* stream);
meta_status meta_plan_destroy(meta_plan* plan);

/* Size of the library's own device scratch used by meta_cost_and_grad_noalloc. */
#define META_NOALLOC_MAX_BYTES (64u << 20)

/* meta_cost_and_grad without a workspace argument.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * themselves.  Examples are code that runs while its stream is being captured
 * into a CUDA graph, where an allocation is not a stream operation and may not
 * be made; plug-ins whose host application owns every device allocation
 * through its own pool; and real-time loops that must never enter the
 * driver's allocator.  The caller passes inputs and outputs only (same
 * meaning as meta_cost_and_grad).
 *
 * The scratch is one fixed array of META_NOALLOC_MAX_BYTES (64 MiB) that every
 * GPU which loads this library holds until the process exits.  A problem whose
 * meta_workspace_size exceeds it is rejected with META_ERR_WORKSPACE before any
 * GPU work; the call itself allocates nothing.  The first call on a device
 * looks up the array's device address (with that device current); make that
 * first call before any stream capture.  Every call uses the same array, which
 * keeps the previous call's contents (its status word is cleared at each call):
 * calls that overlap on the GPU -- from two streams or two threads -- race and
 * corrupt each other, so order them on one stream.  The images and outputs must
 * live on the current device, whose array the call uses.  Faults detected on
 * the device (a bounded wait that ran out) are latched in the array's status
 * word, which meta_noalloc_status reads: check it after a call, before the next
 * call clears it. */
meta_status meta_cost_and_grad_noalloc(const meta_problem* prob, const float* I0, const float* J,
                                       const float* p0, const float* mu, const float* rho,
                                       const float* lambda, double* cost, float* grad,
                                       void* stream);

/* meta_workspace_status for the array of meta_cost_and_grad_noalloc on the
 * current device: the bits latched since the last call began (bit 0: a bounded
 * wait ran out and the call's results are invalid, returned as
 * META_ERR_TIMEOUT; bit 1, information only: an adjoint step transposed the
 * interpolation by the atomic scatter).  Synchronises `stream`; clear != 0
 * resets the word.  Allocates nothing.  (Deployment aid; the paper has no
 * counterpart.) */
meta_status meta_noalloc_status(int clear, void* stream, unsigned int* fault_bits);

/* meta_selftest_timeout on the array of meta_cost_and_grad_noalloc on the
 * current device: a bounded device wait that runs out after limit_ns (in
 * [1 ms, 2 s]) and latches bit 0, which meta_noalloc_status then reports.
 * Nothing faults; the next call clears the word.  (Test aid for the failure
 * detection of callers that cannot allocate; the paper has no counterpart.) */
meta_status meta_noalloc_selftest_timeout(unsigned long long limit_ns, void* stream);

/* Tile shapes of the kernels for one problem shape (ndim, dims, batch,
 * sigma): planes per CTA of the 3-D kernels that march along z (adjoint
 * transport, advect), tile lengths of the strided blur passes along y and z,
 * and the tile width of the x pass.  0 in a field means the built-in choice
 * (extents split into equal tiles of at most 128; a wave-fill heuristic for
 * the plane chunks). */
typedef struct {
    int zc_transport; /* 3-D only; in [1, dims[0]] */
    int zc_advect;    /* 3-D only; in [1, dims[0]] */
    int ly;           /* multiple of 16 in [16, 192], ly + roundup8(2 ceil(3 sigma) + 1) <= 256 */
    int lz;           /* 3-D only; as ly */
    int txw;          /* multiple of 8 in [8, 256] whose staged row txw + 2 hx fits one
                         TMA box of 256 floats; hx, the x halo, is the least multiple
                         of 4 that is >= r + 1, >= r4 and >= kp - r4, with r =
                         ceil(3 sigma), r4 = r rounded up to a multiple of 4 and kp =
                         r4 + r + 1 rounded up to a multiple of 8 (20 for sigma 6) */
    int split;        /* meta_plan_create records the batch as this many sub-batches on
                         parallel graph branches, in [1, min(batch, 16)]; the eager calls
                         ignore it */
} meta_tuning;

/* Autotuner: times meta_cost_and_grad on these inputs (same arguments) for
 * candidate tile shapes (median of nine calls after a warm-up), one field at a
 * time in the order above, in two sweeps; a field moves off its current value
 * only for a candidate at least 1 % faster.  Then it times recorded plans (meta_plan_create) for the batch
 * split, and records the result for the problem shape in a process-wide table
 * that every later call and plan with that shape uses.  No field changes any
 * result: every output is summed in the same order.  Blocking: synchronises
 * `stream` (not capturable); overwrites cost and grad; `out` (may be NULL)
 * receives the choice. */
meta_status meta_autotune(const meta_problem* prob, const float* I0, const float* J,
                          const float* p0, const float* mu, const float* rho, const float* lambda,
                          double* cost, float* grad, void* ws, size_t ws_bytes, void* stream,
                          meta_tuning* out);

/* Tile shapes on disk, a JSON file: {"format": "meta-tuning", "version": 1,
 * "arch": ..., "entries": [{"ndim", "dims", "batch", "sigma", "sigma_bits" (the
 * FP32 bit pattern of sigma; wins over "sigma" when present), "zc_transport",
 * "zc_advect", "ly", "lz", "txw", "split"}, ...]}, other keys ignored.  Files
 * are written to a temporary name and renamed, so readers see whole files.
 * meta_tuning_save: every shape of the process-wide table.  meta_tuning_load:
 * records every entry as meta_tuning_set does; a file with any malformed or
 * out-of-range entry is refused whole (META_ERR_FORMAT, nothing recorded);
 * META_ERR_IO when it cannot be read.  `entries` (nullable) receives the count.
 * meta_tuning_cache: names the cache file of meta_autotune (NULL or "": none)
 * and records the entries it already holds (a missing file is an empty cache).
 * While a cache is named, meta_autotune for a shape that the cache holds
 * records that entry and returns without timing anything (cost and grad are
 * not written), and a new tuning result is merged into the file (entries that
 * other processes wrote meanwhile are kept); META_ERR_IO if that write fails
 * (the result is recorded in the table all the same).  Host only; no call
 * here touches the GPU. */
meta_status meta_tuning_save(const char* path);
meta_status meta_tuning_load(const char* path, int* entries);
meta_status meta_tuning_cache(const char* path, int* entries);

/* The tile shapes a call with this problem uses (tuned, set, or built-in,
 * with 0 fields resolved). */
meta_status meta_tuning_get(const meta_problem* prob, meta_tuning* out);

/* Records tile shapes for the problem shape (tun == NULL: forget them).
 * META_ERR_INVALID_ARG if a field is out of its range or a resulting grid
 * exceeds the launch limits. */
meta_status meta_tuning_set(const meta_problem* prob, const meta_tuning* tun);

/* L-BFGS over the cost of Eq. 4 (the quasi-Newton alternative to the paper's
 * gradient descent, Sec. 3): the inverse-Hessian product by the two-loop
 * recursion (Nocedal & Wright, Algorithm 7.4) over the last m pairs
 * s = x_{k+1} - x_k, y = g_{k+1} - g_k of each instance, H_0 = gamma I with
 * gamma = s^T y / y^T y of the newest usable pair; a pair with s^T y <= 1e-12 y^T y
 * is not used.  Vectors are FP32 [batch, N] (N voxels); dot products are FP64
 * with a fixed summation order.  m in [1, 64].
 * meta_lbfgs_workspace_size: device bytes of the L-BFGS workspace `lws`
 * (256-byte aligned, separate from the cost workspace `ws`). */
meta_status meta_lbfgs_workspace_size(const meta_problem* prob, int m, size_t* bytes);

/* d = -H g for given pairs: s[i], y[i] (device [batch, N], i < npairs <= m,
 * oldest first).  Synchronises the stream (it reads s^T y back). */
meta_status meta_lbfgs_direction(const meta_problem* prob, int m, int npairs,
                                 const float* const* s, const float* const* y, const float* g,
                                 float* d, void* lws, size_t lws_bytes, void* stream);

/* Minimises L(p0) = the sum of the three terms of Eq. 4 per instance, starting
 * from p0 (device, overwritten by the last accepted iterate).  Each iteration:
 * the direction d = -H g (or d = -h0 g / max|g| without a usable pair, or when
 * -H g does not descend, which also forgets the instance's pairs), then a
 * backtracking line search from step 1, halving up to 12 times, that accepts
 * the first step a with L(x + a d) <= L(x) + 1e-4 a g^T d.  An instance whose
 * search fails, or whose gradient is zero (d = 0), keeps its iterate and stops.  cost_hist (host, nullable):
 * [iters + 1][batch] costs, entry 0 at the start; iters_done (host, nullable):
 * [batch] the last iteration that moved each instance.  Blocks the host: the
 * costs of every trial are read back.  ws: a cost workspace (meta_workspace_size). */
meta_status meta_lbfgs_minimize(const meta_problem* prob, const float* I0, const float* J,
                                float* p0, const float* mu, const float* rho,
                                const float* lambda, int iters, int m, float h0, void* ws,
                                size_t ws_bytes, void* lws, size_t lws_bytes, double* cost_hist,
                                int* iters_done, void* stream);

/* Continues a minimisation for `iters` more iterations from the state that the
 * last meta_lbfgs_minimize / meta_lbfgs_resume on this lws ended with (or that
 * meta_lbfgs_state_load put there): the iterate p0 (which must hold that run's
 * last accepted iterate), its gradient, the m pairs, the costs and stopped
 * flags.  The same sequence of iterates results as one longer run, bit for bit.
 * cost_hist: [iters + 1][batch], entry 0 the cost at the resume point;
 * iters_done counts iterations across the runs.  META_ERR_FORMAT if lws holds
 * no finished run (the state is valid only after a run returned META_OK). */
meta_status meta_lbfgs_resume(const meta_problem* prob, const float* I0, const float* J,
                              float* p0, const float* mu, const float* rho, const float* lambda,
                              int iters, int m, float h0, void* ws, size_t ws_bytes, void* lws,
                              size_t lws_bytes, double* cost_hist, int* iters_done,
                              void* stream);

/* Host save / resume of the L-BFGS state (the paper has none: its optimiser
 * runs once, Sec. 3).  The host image is an 80-byte header (tag "METALBFS",
 * u32 version 1, i32 ndim, dims[3] (0 past ndim), batch, m, iterations done,
 * pairs held, ring head, two zero words, then u64 voxels per instance, payload
 * bytes and the FNV-1a 64-bit checksum of the payload; little-endian),
 * then the gradient [batch, N] f32, the pair rings S and Y [m][batch, N] f32,
 * rho [m][batch] f64, gamma [batch] f64, the costs [batch] f64 and the stopped
 * and last-moved flags [batch] i32.  p0 is not part of it: save the iterate
 * with it.
 * meta_lbfgs_state_size: bytes of the image.
 * meta_lbfgs_state_check (host only): META_OK when `host` is an intact image
 * for this problem and m, META_ERR_FORMAT when it is not (size, tag, version,
 * shape, ring indices or checksum).
 * meta_lbfgs_state_save: writes the image of the state in lws (META_ERR_FORMAT
 * if lws holds no finished run).  meta_lbfgs_state_load: checks the image, then
 * copies it into lws for meta_lbfgs_resume.  Both synchronise `stream`; the
 * host buffer is the caller's and is not kept. */
meta_status meta_lbfgs_state_size(const meta_problem* prob, int m, size_t* bytes);
meta_status meta_lbfgs_state_check(const meta_problem* prob, int m, const void* host,
                                   size_t host_bytes);
meta_status meta_lbfgs_state_save(const meta_problem* prob, int m, const void* lws,
                                  size_t lws_bytes, void* host, size_t host_bytes, void* stream);
meta_status meta_lbfgs_state_load(const meta_problem* prob, int m, const void* host,
                                  size_t host_bytes, void* lws, size_t lws_bytes, void* stream);

/* Gradient descent on the cost of Eq. 4, the paper's optimiser (Sec. 3), with
 * the step normalised per instance: p0 <- p0 - h0 g / max|g| (no step where
 * g = 0), `iters` steps.  Its whole state is the iterate p0 and the number of
 * steps taken, so a run of a + b steps equals a run of a steps followed by one
 * of b (bit for bit).  lws: an L-BFGS workspace for m = 1.  cost_hist (host,
 * nullable): [iters + 1][batch], the cost of every iterate; with it the host
 * reads the costs once per step, without it the host does not wait between
 * steps.  Synchronises `stream` before returning. */
meta_status meta_gd_minimize(const meta_problem* prob, const float* I0, const float* J,
                             float* p0, const float* mu, const float* rho, const float* lambda,
                             int iters, float h0, void* ws, size_t ws_bytes, void* lws,
                             size_t lws_bytes, double* cost_hist, void* stream);

/* Device-side status word latched in ws since it was last cleared.  Bit 0: a
 * bounded TMA wait ran out (the call's results are invalid; returns
 * META_ERR_TIMEOUT).  Bit 1 (information only): an adjoint step had per-step
 * displacements beyond the deterministic gather window (8 voxels or more in
 * 2-D, 4 or more in 3-D) and transposed the interpolation by an atomic scatter
 * instead, so its summation order is not fixed.  Bit 2 (only in the
 * bounds-checked debug build, libmeta_check.so, compiled with
 * META_CHECK_BOUNDS): an index the kernels computed from the data (the lower
 * corner of a foot, a record cell decoded by a transport) left its range; it was
 * clamped, so nothing outside its buffer was read or written, but the call's
 * results are invalid.  Synchronises `stream`.  clear != 0 resets it. */
meta_status meta_workspace_status(void* ws, size_t ws_bytes, int clear, void* stream,
                                  unsigned int* fault_bits);

/* Self-test of device-side failure detection: enqueues one small kernel that
 * waits, exactly as the blur kernels wait for their TMA tiles, on an mbarrier
 * armed for bytes that never arrive, with the bound limit_ns (in [1 ms, 2 s])
 * instead of the 2 s of the real waits.  The wait runs out and latches bit 0 in
 * the status word of ws, which meta_workspace_status then reports as
 * META_ERR_TIMEOUT; nothing faults, the context stays usable, and clearing the
 * word restores the workspace. */
meta_status meta_selftest_timeout(void* ws, size_t ws_bytes, unsigned long long limit_ns,
                                  void* stream);

/* Tracing (the paper has none): every meta_cost_and_grad, and every call and
 * plan recording built on it, marks its phases as NVTX ranges on the calling
 * host thread: "meta.cost_and_grad" around "meta.forward" (the T steps of
 * Eq. 3), "meta.cost" (Eq. 4) and "meta.adjoint" (the reverse sweep), which
 * holds one "meta.recompute" per checkpoint segment re-run from its stored
 * state (none with every state kept).  Ranges bracket the enqueueing of each
 * phase's kernels (profilers such as ncu --nvtx attribute kernels to them);
 * they cost a few hundred nanoseconds when no tool is attached.
 * meta_trace_set: a host callback (NULL: none) that receives the same pushes
 * (push = 1) and pops (push = 0) with the range's name (a static string) and
 * `user`, on the thread that makes the call; it must not call into this
 * library.  meta_trace_selftest: pushes "meta.selftest", pushes and pops
 * "meta.selftest.inner", pops "meta.selftest" (host only, for checking a
 * callback or a tool). */
typedef void (*meta_trace_fn)(const char* name, int push, void* user);
meta_status meta_trace_set(meta_trace_fn fn, void* user);
meta_status meta_trace_selftest(void);

/* Human-readable name of a status code (static string). */
const char* meta_status_string(meta_status s);

/* Kernel classes reported by the timer below. */
enum {
    META_K_PACK = 0,       /* copy I0, p0 into the pitched trajectory */
    META_K_XPASS_M,        /* m = p grad I fused with the x pass of K */
    META_K_STRIDED_FWD,    /* y (and z) passes of K in the forward step */
    META_K_ADVECT,         /* backtrack + interpolate + momentum/intensity update */
    META_K_COST,           /* Eq. 4 partial sums and their final reduction */
    META_K_ADJ_INIT,       /* adjoint start from gI1, gp1 */
    META_K_ADJ_PRE,        /* pointwise part of the adjoint step */
    META_K_ADJ_GATHER,     /* gather-form transpose of the interpolation, v^ */
    META_K_XPASS_ADJ,      /* x pass of K on v^ */
    META_K_STRIDED_ADJ,    /* y (and z) passes of K on v^ */
    META_K_ADJ_GRADP,      /* transpose of m = p grad I */
    META_K_UNPACK,         /* copy I_T, p_T out */
    META_K_DEFORM,         /* one step of the deformation phi_{t+1} = phi_t o (Id - dt v_t) */
    META_K_DEFORM_OUT,     /* phi_T - Id and det D phi_T out */
    META_K_ADJ_JAC,        /* META_P_UPDATE_DET: the higher-order part of the adjoint of det */
    META_K_EULER,          /* Eulerian or hybrid step (META_SCHEME_EULER / _HYBRID) */
    META_K_COUNT
};

/* Profiling aid, off by default, not thread-safe: after meta_timer_start(cap)
 * every kernel launched by the calls above (up to cap launches) is bracketed
 * by a pair of CUDA events on the call's stream.  meta_timer_stop()
 * synchronises those events, writes per kernel class (arrays of META_K_COUNT)
 * the summed device milliseconds and the number of launches, and turns the
 * timer off.  The events are host objects created by meta_timer_start. */
meta_status meta_timer_start(int cap);
meta_status meta_timer_stop(float* ms_per_class, int* launches_per_class);
const char* meta_kernel_name(int kernel_class);

#ifdef __cplusplus
}
#endif

#endif /* META_H */
