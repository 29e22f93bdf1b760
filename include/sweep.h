/*
 * sweep.h -- C ABI of the B300 swept-rule solver for explicit 2D stencil PDEs.
 *
 * The solver advances a periodic 2D field with the two-dimensional swept
 * rule (Walker & Niemeyer, Sec. 3.3): each block of the grid is taken through
 * Up-Pyramid, X/Y-Bridge, Octahedron and Down-Pyramid phases, advancing as
 * many RK stages on chip as its dependency cone allows before its edges go
 * back to device memory.  A conventional one-kernel-per-step solver
 * ("Standard", Sec. 3.1) gives the same result bit for bit.
 *
 * Equations (time rule: explicit midpoint RK2 unless set otherwise):
 *   SWEEP_HEAT  -- T_t = alpha (T_xx + T_yy), 5-point Laplacian (App. A).
 *                  State: 1 component.  Stencil radius per stage n = 1.
 *   SWEEP_EULER -- compressible Euler, ideal gas (App. B): pressure-ratio
 *                  minmod reconstruction, Rusanov-form flux.
 *                  State: 4 components (rho, rho u, rho v, E).  n = 2.
 *
 * Conventions shared by every entry point:
 *   - All arithmetic is IEEE binary64.
 *   - State layout: structure of arrays [ncomp][ny][nx], x fastest,
 *     contiguous, base address 16-byte aligned.  Periodic in x and y.
 *     Cell (i, j) of the heat problem sits at x = i dx, y = j dx; the Euler
 *     problem stores cell averages.  dy = dx.
 *   - Ownership: the state and the workspace are device memory owned by the
 *     caller (e.g. torch tensors).  The handle owns host-side tables only.
 *     No entry point allocates device memory.
 *   - Streams: work is enqueued on the given stream (a cudaStream_t; NULL
 *     is the legacy default stream) and the call returns without waiting,
 *     like a CUDA library call.  Launch-configuration errors are reported by
 *     the return code; a fault during execution surfaces at the caller's
 *     next synchronisation.  No entry point synchronises the device unless
 *     its comment says so, so the enqueued sequence can be captured into a
 *     CUDA graph.
 *   - Errors: a nonzero sweep_status; nothing aborts, exits or traps.
 *     Argument and launch errors are returned at once.  What the kernels
 *     find while they run goes to a device error word, the first 4 bytes
 *     of the workspace header, which every run clears on entry: bit
 *     SWEEP_DEV_NONFINITE (a value of a run's final state was an infinity
 *     or a NaN, e.g. after a time step beyond the CFL bound), and, in the
 *     checked build libsweep_checked.so only, bit SWEEP_DEV_LAUNCH (a kernel
 *     found its grid, block or shared memory wrong for its geometry; it
 *     then does nothing).
 *     sweep_check reads it; with the "check" parameter set every run reads
 *     it before returning (and so waits for the GPU).
 *   - Threads: one handle must not be used from two threads at once;
 *     separate handles are independent.
 */
#ifndef SWEEP_H
#define SWEEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* the type behind cudaStream_t */

typedef struct sweep_s sweep_t; /* opaque solver handle */

enum sweep_eqn { SWEEP_HEAT = 0, SWEEP_EULER = 1 };

enum sweep_status {
    SWEEP_OK = 0,
    SWEEP_EINVAL = 1,      /* bad argument or geometry                       */
    SWEEP_ENOMEM = 2,      /* host allocation failed                         */
    SWEEP_ECUDA = 3,       /* a CUDA call or kernel launch failed            */
    SWEEP_ETIMEOUT = 4,    /* reserved for a bounded device-side wait that gives
                              up; no kernel of this build waits on another CTA
                              (clusters use the hardware cluster barrier), so no
                              call returns it                                 */
    SWEEP_EUNSUPPORTED = 5, /* valid request that this build does not handle */
    SWEEP_EDEVICE = 6      /* the device error word was set (sweep_check)    */
};

/* bits of the device error word */
#define SWEEP_DEV_LAUNCH 1u
#define SWEEP_DEV_NONFINITE 2u

/*
 * Create a solver for an nx x ny periodic grid.
 *   eqn    SWEEP_HEAT or SWEEP_EULER.
 *   dt, dx time step and cell size (dy = dx); heat uses r = alpha dt / dx^2.
 *   tile   block edge b of the swept decomposition (Sec. 3.2): even,
 *          b > 2n, nx % b == 0, ny % b == 0, nx/b >= 2, ny/b >= 2.
 *   depth  stage-levels per swept phase d: 2 <= d <= k = b/(2n) - 1 (Eq. 1),
 *          d even so that every phase ends on a whole RK2 step; 0 picks the
 *          largest even d allowed.
 * Defaults: alpha = 1, gamma = 1.4, limiter 0, RK2.  The Standard solver
 * uses its own block edge ("standard_tile"): by default the first of the
 * list that divides the grid into at least its minimum number of blocks --
 * heat: 64 (1024 blocks), 32 (1024), then 16, 8, 24, 12, 48, 40, 20, 10
 * (148 each, one per SM of a B300); Euler: 16, 8, 24, 12, 64, 48, 40, 20,
 * 10 (148 each) -- else the allowed edge of that list giving the most
 * blocks, else the smallest even edge in [8, 64] that divides both sides.  On success *out receives the handle (destroy with
 * sweep_destroy).  Returns SWEEP_EINVAL for any violated bound.
 */
int sweep_create(int eqn, int64_t nx, int64_t ny, double dt, double dx, int tile, int depth,
                 sweep_t **out);

/*
 * Set a scalar parameter.  Keys:
 *   "alpha"          heat diffusivity (> 0)
 *   "gamma"          ratio of specific heats (> 1)
 *   "limiter"        0 pressure-ratio minmod, textbook orientation (App. B,
 *                    reading of the garbled ratio); 1 the orientation as printed;
 *                    2 no limiting (face value = average of the two cells; not
 *                    a scheme of the paper: a smooth variant for checking the
 *                    adjoint against finite differences)
 *   "scheme"         heat time rule: 0 RK2 midpoint, 1 forward Euler (App. A)
 *   "standard_tile"  block edge of the Standard solver (8..64, divides nx, ny)
 *   "cluster"        CTAs sharing one swept window through distributed shared
 *                    memory, for every swept kernel (1, 2, 4); "cluster_oct"
 *                    and "cluster_bridges" set the Up-Pyramid/Octahedron and
 *                    the Bridge kernels separately.  Defaults: heat 1 and 1;
 *                    Euler 2 and 1 while 2 CTAs per block fit one per SM of a
 *                    B300 (at most 74 blocks), else 1 and 1.  A size whose
 *                    shared memory does not fit is rejected.
 *   "passes"         row bands each CTA takes one after another per level
 *                    (1, 2, 4): less shared memory per CTA, more CTAs per SM
 *   "profile"        1: every later run brackets each kernel launch with a
 *                    pair of CUDA events on its stream (read them with
 *                    sweep_profile_read); 0 (default): no events
 *   "l2_fetch_bytes" 32, 64 or 128: set, at once, the L2 fetch granularity
 *                    limit (cudaLimitMaxL2FetchGranularity) of the calling
 *                    process's CUDA context on the current device -- it
 *                    applies to every kernel of the process until changed,
 *                    and ends with the process.  The level store's thin
 *                    column pieces use one 32-byte sector of each 128-byte
 *                    line; with 32 the swept kernels' DRAM reads drop to the
 *                    bytes they use (heat, block 64, depth 30: 2.5x -> 1.0x
 *                    per launch; run time unchanged, the kernels being bound
 *                    by FP64 issue).  0 (default): the context is not touched.
 *                    Returns SWEEP_ECUDA if the limit cannot be set.
 *   "check"          1: every run (swept, standard, adjoint, static) ends
 *                    by waiting for its stream and reading the device error
 *                    word, and returns SWEEP_EDEVICE if a bit is set (the
 *                    run is then not capturable into a CUDA graph); 0
 *                    (default): runs stay asynchronous
 * Returns SWEEP_EINVAL for an unknown key or a value out of range.
 */
int sweep_set_param(sweep_t *h, const char *key, double value);

/* Read back a parameter (the keys above plus "tile", "depth", "r",
 * "nx", "ny", "ncomp", "radius").  Returns SWEEP_EINVAL for an unknown key. */
int sweep_get_param(const sweep_t *h, const char *key, double *value);

/*
 * Bytes of device workspace that sweep_run_swept and sweep_run_standard need
 * (256-byte aligned base): (depth + 1) level slots of one state each plus a
 * small header.  The Standard solver needs only the first slot.
 */
size_t sweep_workspace_bytes(const sweep_t *h);

/*
 * Advance d_state (device, [ncomp][ny][nx] fp64) in place by exactly nsteps
 * time steps with the swept rule (Sec. 3.3): Up-Pyramid, then
 * [Bridges, Octahedron] cycles with the block grid shifted by b/2 each
 * cycle, then Bridges and Down-Pyramid; the 2*nsteps mod depth stage-levels
 * that do not fill a cycle are taken as Standard steps.  Bit-identical to
 * sweep_run_standard.  d_ws: caller-owned device workspace of
 * sweep_workspace_bytes(h) bytes, 256-byte aligned; its contents on entry
 * do not matter.  nsteps >= 0.
 */
int sweep_run_swept(sweep_t *h, double *d_state, int64_t nsteps, void *d_ws,
                    struct CUstream_st *stream);

/*
 * Advance d_state in place by nsteps with the Standard solver (Sec. 3.1):
 * one kernel per RK2 step, each block loading its tile plus a 2n halo,
 * taking stage 1 on the tile plus an n halo and stage 2 on the tile.
 */
int sweep_run_standard(sweep_t *h, double *d_state, int64_t nsteps, void *d_ws,
                       struct CUstream_st *stream);

/*
 * Gradient of a final-state loss with respect to the initial state (the
 * discrete adjoint; reverse mode of the explicit scheme, which the swept
 * rule only reorders, Sec. 3.3).  d_lamT = dL/dQ^N (device, state layout);
 * on return d_lam0 = dL/dQ^0.  At the limiter's switches, the max of the
 * wave speeds and |u_n| the derivative of the branch the forward step took
 * is used.
 *   heat:  the step is linear with a symmetric 5-point operator, so the
 *          adjoint step is again a two-stage stencil update
 *          (mu* = r t(lam), lam_n = fma(r/2, t(mu*), lam + mu*)) and runs
 *          through the swept kernels.  d_q0 is not read (may be NULL);
 *          d_lam0 may equal d_lamT.
 *   Euler: a forward swept pass from d_q0 keeps a checkpoint every
 *          ckpt_every steps; each segment is then recomputed by one swept
 *          run from its checkpoint that records every step's state and
 *          first stage (the steps after its last whole swept cycle are
 *          Standard steps), and reversed step by step: face-wise reverse
 *          mode of the flux, gathered per cell in a fixed order (x faces,
 *          then y faces, in increasing face index); the terms that
 *          neighbouring faces share, and the reverse of each cell's
 *          pressure, are computed once per cell.  d_lam0 must not alias
 *          d_lamT.
 * d_ws: sweep_adjoint_workspace_bytes(h, nsteps, ckpt_every) bytes,
 * 256-byte aligned.  Asynchronous on the stream like the other runs.
 */
size_t sweep_adjoint_workspace_bytes(const sweep_t *h, int64_t nsteps, int ckpt_every);
int sweep_adjoint(sweep_t *h, const double *d_q0, const double *d_lamT, double *d_lam0,
                  int64_t nsteps, int ckpt_every, void *d_ws, struct CUstream_st *stream);

/*
 * Batched swept runs: advance d_states[i] (device, each in its instance's
 * layout) in place by nsteps[i] with handle hs[i], for i < count.  The
 * instances are independent and may differ in equation, size, tile, depth
 * and cluster settings.  Each instance's launch sequence goes to one of a
 * pool of internal streams (largest work first), forked from `stream` and
 * joined back into it by events: the instances overlap on the GPU and the
 * whole batch can be captured from `stream` into one CUDA graph.  The first
 * call on a device creates the stream pool (make it before any capture).
 * d_ws: sweep_batch_workspace_bytes(hs, count) bytes, 256-byte aligned,
 * carved into one region per instance.  Each result is bit-identical to
 * that instance's sweep_run_swept.  A handle must appear once per batch.
 */
size_t sweep_batch_workspace_bytes(sweep_t *const *hs, int count);
int sweep_batch_run(sweep_t *const *hs, double *const *d_states, const int64_t *nsteps, int count,
                    void *d_ws, struct CUstream_st *stream);

/*
 * Allocation-free form of sweep_run_swept (the paper has no counterpart;
 * this is an interface convenience).
 *
 * For callers that cannot allocate device memory when they advance a state,
 * e.g. a plug-in inside an application that owns all GPU memory through its
 * own pool, or a latency-critical loop where an allocation or its failure
 * mid-run is not acceptable.  Instead of a caller workspace, the level store
 * lives in a fixed device array of SWEEP_STATIC_SCRATCH_BYTES inside the
 * library.  Every GPU on which the library is loaded holds that array until
 * the process exits.
 *
 *   - Same arguments and result as sweep_run_swept minus d_ws.  The state is
 *     still caller-owned device memory, and the current device must be the
 *     device of the state and the stream.
 *   - Returns SWEEP_EINVAL when sweep_workspace_bytes(h) exceeds
 *     SWEEP_STATIC_SCRATCH_BYTES (e.g. Euler 256 x 256 at depth 6 needs
 *     14 MiB and fits; heat 1024 x 1024 at depth 14 needs 120 MiB and does
 *     not), and SWEEP_EUNSUPPORTED while "profile" is on.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it.  Make that first call before
 *     any stream capture.
 *   - All calls share the one array, which keeps what the last call left
 *     there.  Nothing in it needs to start at zero: a swept run writes every
 *     value of the level store before reading it.  Calls that overlap on the
 *     GPU (on any streams of the same device) race on the array and give
 *     wrong results; serialise them.
 */
#define SWEEP_STATIC_SCRATCH_BYTES ((size_t)16 << 20)
int sweep_run_swept_static(sweep_t *h, double *d_state, int64_t nsteps,
                           struct CUstream_st *stream);

/*
 * Per-kernel device time of the launches recorded since "profile" was set
 * or since the last read.  Kinds: 0 Up-Pyramid, 1 Bridges, 2 Octahedron,
 * 3 Down-Pyramid, 4 Standard step.  ms[k] receives the summed event time of
 * kind k and launches[k] the number of its launches, for k < nkinds.  Waits
 * for the recorded events (synchronises with the stream they were recorded
 * on).  Returns SWEEP_ECUDA if an event cannot be read.
 */
int sweep_profile_read(sweep_t *h, double *ms, int64_t *launches, int nkinds);

/*
 * FP64 throughput probe (a measuring instrument, not part of the method):
 * launches `blocks` CTAs of `threads` threads on the stream; every thread
 * takes 8 independent chains of `iters` fused multiply-adds and writes one
 * double to d_out[blocks * threads] (device, caller-owned).  The launch does
 * 16 * iters * blocks * threads flops (an fma counts 2); timed with events on
 * the stream it gives the FP64 rate that bounds the swept kernels.
 * Returns SWEEP_EINVAL for threads not a multiple of 32 in [32, 1024].
 */
int sweep_fp64_probe(double *d_out, int64_t iters, int blocks, int threads,
                     struct CUstream_st *stream);

/*
 * Wait for `stream`, read the device error word of the workspace d_ws (the
 * workspace of the runs to check, 256-byte aligned), store it in *bits (if
 * bits is not NULL) and clear it.  Returns SWEEP_OK when no bit was set,
 * SWEEP_EDEVICE when one was, SWEEP_ECUDA if the wait or the copy failed.
 * Synchronous.  For a batch, each instance's word heads its own region of
 * the batch workspace.
 */
int sweep_check(const void *d_ws, unsigned *bits, struct CUstream_st *stream);

/*
 * Test hooks: host-side fault injection.  sweep_inject_fault(site, n) makes
 * the n-th next pass through `site` fail the way the real failure would
 * (n = 0, or site 0, disarms):
 *   SWEEP_SITE_HOST_ALLOC   the handle allocation of sweep_create
 *                           (sweep_create returns SWEEP_ENOMEM)
 *   SWEEP_SITE_STREAM_POOL  creating a stream or an event of the batch
 *                           pool (sweep_batch_run returns SWEEP_ECUDA and
 *                           destroys what it had created)
 *   SWEEP_SITE_EVENTS       creating a profiling event pair (that launch is
 *                           not timed)
 * Nothing here makes a GPU fault.  The setting is process-wide; returns
 * SWEEP_EINVAL for an unknown site or a negative n.
 * sweep_live_cuda_objects() counts the CUDA streams and events the library
 * holds (the batch pools and the profiling events of live handles).
 */
enum sweep_fault_site {
    SWEEP_SITE_HOST_ALLOC = 1,
    SWEEP_SITE_STREAM_POOL = 2,
    SWEEP_SITE_EVENTS = 3
};
int sweep_inject_fault(int site, int nth);
int sweep_live_cuda_objects(void);

/* Release a handle (NULL is ignored). */
void sweep_destroy(sweep_t *h);

/* Static description of a status code. */
const char *sweep_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* SWEEP_H */
