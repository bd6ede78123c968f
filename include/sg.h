/*
 * sg.h -- C ABI of libsg, a GB300 (sm_103a) library for Metropolis aging dynamics of mean-field
 * spin glasses after a quench (arXiv:1906.11195, "Strong ergodicity breaking in aging of mean
 * field spin glasses").
 *
 * Models
 *   Viana-Bray (VB):  H = -sum_{(ij) in E} J_ij s_i s_j on a sparse graph, J_ij = +-1 (Eq. 3).
 *                     64 disorder samples ("lanes") share one graph, each with its own couplings
 *                     and initial spins, packed one bit per lane in 64-bit words (multispin
 *                     coding, SI section 2 and the caption of Table 1).
 *   Sherrington-Kirkpatrick (SK): H = -sum_{i<j} J_ij s_i s_j / sqrt(N), J_ij = +-1 (Eq. 1 with
 *                     the binary couplings of SI section 1).  R replicas share J.
 * Dynamics: single-spin-flip Metropolis at fixed temperature from a random start (Methods; SI
 * sections 1-2).  Time unit = one sweep (every spin visited once).  VB visits one graph colour
 * class at a time (the independent-set update of SI section 3, generalised from the bipartite
 * halves to a greedy colouring); SK visits i = 0..N-1 in order (SI section 1, "fixed order").
 * Observables (integer counts; divide by N): two-time correlation C(t_w+t, t_w) = sum_i
 * s_i(t_w+t) s_i(t_w) (the definition after Eq. 1 and Eq. formula1), the overlap of replica
 * pairs (2p, 2p+1) (the "two clones" of SI section 1), and the energy.
 *
 * Random numbers (the paper names none): Philox4x32-10, key = (seed_lo, seed_hi).
 *   update draw of replica r, sweep t (0-based), vertex i: word (r mod 4) of counter (i, t, r/4, 0)
 *   initial spins of replica r, vertex i: lane bits = w0 | w1 << 32 of counter (i, 0, r, 1),
 *   bit = 1 means s = -1 (SK uses lane bit 0).  One draw is shared by the 64 lanes of a word.
 * Acceptance: flip iff dE <= 0 or r32 < thr(dE), thr = min(2^32-1, floor(2^32 exp(-dE/T))) in
 * double precision; VB dE = 2m with m = s_i sum_j J_ij s_j, thr[m] = f(-2.0*beta*m);
 * SK dE = 2k/sqrt(N), thr[k] = f(-(2.0*beta*k)/sqrt((double)N)), beta = 1.0/T.
 * Results are bit-exact functions of (instance, temperatures, seed, schedule): the kernel choice,
 * block size and launch shapes never change them.
 *
 * Memory and ownership
 *   - Host arrays passed to sg_create_* are read during the call only; the caller keeps them.
 *   - The library allocates no device memory.  The caller allocates one device workspace of
 *     sg_workspace_bytes() bytes (e.g. a PyTorch uint8 tensor) and lends it through sg_attach()
 *     until sg_destroy(); it must be 256-byte aligned.
 *   - The CUDA stream given to sg_attach() is borrowed; all device work of the handle is queued
 *     on it.  Calls on one handle must not overlap from several host threads.
 * Errors: every call returns SG_OK (0) or a negative code; sg_last_error() gives a message for
 * the calling thread.  No C++ exception crosses this interface.
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SG_OK 0
#define SG_EINVAL (-1)   /* bad argument or instance (asymmetric J, self-loop, bad schedule...) */
#define SG_ENOMEM (-2)   /* workspace too small or misaligned, or host allocation failed */
#define SG_ECUDA (-3)    /* CUDA runtime error; the message names the call */
#define SG_ETIMEOUT (-4) /* a bounded device-side wait expired; the handle must be destroyed */
#define SG_ESTATE (-5)   /* call out of order (e.g. sweep before attach) */

/* kernel selection */
#define SG_VB_PLAIN 0    /* baseline: one thread per (vertex, lane, replica), int8 spins, CSR */
#define SG_VB_PACKED 1   /* 64 lanes per uint64, bit-sliced field count, sliced-ELL graph */
#define SG_SK_PLAIN 2    /* baseline: sequential order, one thread block per replica */
#define SG_SK_BLOCKED 3  /* blocked sweep: in-block update + tensor-core off-block field update */

#define SG_VB_MAX_DEGREE 63      /* VB vertex degree limit */
#define SG_VB_MAX_N ((1 << 26) - 1) /* VB vertices per graph */

typedef struct sg_ctx *sg_handle;

/* One Viana-Bray graph with 64 coupling sets (Eq. 3; SI section 2).
 *   n         number of vertices, 2 <= n <= SG_VB_MAX_N
 *   row_ptr   int32[n+1] CSR row offsets (host)
 *   col       int32[row_ptr[n]] neighbour lists (host); simple undirected graph: symmetric, no
 *             self-loop, no duplicate, degree <= SG_VB_MAX_DEGREE
 *   jbits     uint64[row_ptr[n]] couplings per directed entry (host): bit k = 1 iff J_ij = -1
 *             in lane k; the entries (i,j) and (j,i) must hold the same word
 *   seed      Philox key of this graph's random numbers
 *   temps     double[n_replicas] temperatures of the replicas (host); 0 and +inf are allowed */
typedef struct {
    int32_t n;
    const int32_t *row_ptr;
    const int32_t *col;
    const uint64_t *jbits;
    uint64_t seed;
    const double *temps;
} sg_vb_graph;

/* Message of the last failed call on this thread ("" if none).  Owned by the library.
 * Library service; the paper has no counterpart. */
const char *sg_last_error(void);

/* Create a batch of Viana-Bray instances that evolve in lock-step (one sweep of the batch =
 * one sweep of every graph; the batched persistent form of the uneven workloads).
 * Defines: the VB model of Eq. 3 on its graph with 64 coupling sets per word (SI section 2,
 * Table 1), quenched from a random configuration (Methods); the many sizes of Table 1 run as
 * one batch.
 *   graphs[n_graphs]  the instances (host)
 *   n_lanes           lanes reported in the results, 1..64 (the packed kernel always simulates
 *                     all 64; the plain kernel simulates only these)
 *   n_replicas        R >= 1 replicas per graph (R <= 4 for SG_VB_PACKED)
 *   kernel            SG_VB_PLAIN or SG_VB_PACKED (SG_VB_PLAIN requires n_graphs == 1)
 *   tw[n_tw]          strictly increasing snapshot times t_w >= 0 (sweeps)
 *   tm[n_tm]          strictly increasing measurement times >= 0 (sweeps)
 *   out               receives the handle; nothing is on the device until sg_attach()
 * Host-side work: validation, greedy colouring (vertex order), relabelling of each graph into
 * colour classes, construction of the device layout. */
int sg_create_vb(const sg_vb_graph *graphs, int32_t n_graphs, int32_t n_lanes,
                 int32_t n_replicas, int32_t kernel, const int64_t *tw, int32_t n_tw,
                 const int64_t *tm, int32_t n_tm, sg_handle *out);

/* Create an SK instance (Eq. 1 with binary couplings; SI section 1: fixed-order Metropolis,
 * R replicas sharing J, the "two clones" of the overlap).
 *   n          spins, 2 <= n <= 32768
 *   J          int8[n*n] row-major couplings (host): +-1 off the diagonal, 0 on it, symmetric
 *   n_replicas R >= 1 replicas sharing J (a multiple of 16 for SG_SK_BLOCKED)
 *   temps      double[R] replica temperatures (host)
 *   seed       Philox key
 *   kernel     SG_SK_PLAIN or SG_SK_BLOCKED
 *   block      spins per block B for SG_SK_BLOCKED: 64, 128, 256 or 512, or 0 to let the
 *              autotuner choose at attach among 64, 128, 256 and, for n >= 2048, 512 (n is
 *              then padded to a multiple of 512, else of 256); ignored by SG_SK_PLAIN
 *   tw, tm     schedule, as for sg_create_vb */
int sg_create_sk(int32_t n, const int8_t *J, int32_t n_replicas, const double *temps,
                 uint64_t seed, int32_t kernel, int32_t block, const int64_t *tw, int32_t n_tw,
                 const int64_t *tm, int32_t n_tm, sg_handle *out);

/* One SK sample of a batch: n spins, couplings J (int8[n*n], host, as for sg_create_sk), its own
 * Philox key and the temperatures of its n_replicas replicas (double[n_replicas], host). */
typedef struct {
    int32_t n;
    const int8_t *J;
    uint64_t seed;
    const double *temps;
} sg_sk_sample;

/* Create a batch of independent SK samples of uneven size (the uneven-N runs used for the
 * extrapolation in N of SI section 1) that advance in lock-step; each sweep is one CUDA graph
 * whose branches, one per sample, run concurrently.  Arguments as for sg_create_sk; every sample
 * has n_replicas replicas.  block = 0 lets an autotuner pick B per sample, as for sg_create_sk,
 * by timing trial sweeps at attach (the trajectory does not depend on B).  Results are laid out
 * with n_inst = n_samples; spins concatenate int8[R][n_s] over the samples. */
int sg_create_sk_batch(const sg_sk_sample *samples, int32_t n_samples, int32_t n_replicas,
                       int32_t kernel, int32_t block, const int64_t *tw, int32_t n_tw,
                       const int64_t *tm, int32_t n_tm, sg_handle *out);

/* Replace the measurement schedule: tw[n_tw] snapshot times and tm[n_tm] measurement times,
 * each strictly increasing, >= 0 and < 2^32 (as for sg_create_vb).  Before sg_attach any sizes
 * are allowed (the workspace size follows them).  After sg_attach the schedule can still be
 * replaced while no scheduled time has been reached yet (no snapshot or measurement taken,
 * including those at tau = 0) if n_tw and n_tm stay the same (the workspace layout is fixed at
 * attach) and every new time is later than the current tau; otherwise SG_ESTATE.  Bad arrays:
 * SG_EINVAL.  Defines: the waiting times t_w and the log-spaced measurement times t_w + t of
 * the aging protocol (main text, Fig. 1; SI section 3). */
int sg_set_schedule(sg_handle h, const int64_t *tw, int32_t n_tw, const int64_t *tm,
                    int32_t n_tm);

/* Device workspace size the handle needs (bytes).  Library service; no counterpart in the
 * paper. */
int sg_workspace_bytes(sg_handle h, size_t *bytes);

/* Bind the caller's device workspace and CUDA stream (cudaStream_t, may be NULL for the legacy
 * default stream), copy the instance to the device, draw the initial spins (tau = 0) and take the
 * tau = 0 snapshot/measurement if scheduled.  Returns after the copies have completed.
 * Defines: the quench, a random initial configuration at t = 0 (Methods). */
int sg_attach(sg_handle h, void *dev_workspace, size_t bytes, void *cuda_stream);

/* Advance by n >= 0 sweeps, asynchronously on the handle's stream.  Snapshots and measurements
 * due at the times passed are taken on the device on the way.
 * Defines: one sweep = one Metropolis visit of every spin, the time unit of every figure
 * (Methods; SI sections 1-3: colour classes for VB, the fixed order for SK). */
int sg_sweep(sg_handle h, int64_t n);

/* Current time tau (completed sweeps), as queued.  The paper's t, in sweeps (Methods). */
int sg_time(sg_handle h, int64_t *tau);

/* Wait for the handle's queued work; reports device-side errors (SG_ECUDA, SG_ETIMEOUT).
 * Library service; no counterpart in the paper. */
int sg_synchronize(sg_handle h);

/* Shapes of the result arrays: n_inst, n_replicas, n_lanes, n_tw, n_tm (5 int32).
 * Library service; no counterpart in the paper. */
int sg_result_shape(sg_handle h, int32_t *shape5);

/* Copy the scheduled measurements to the host (synchronises).  Defines: C(t_w + t, t_w) as in
 * Eq. formula1 (the sum after Eq. 1), the overlap of the two clones (SI section 1), and the energy
 * of Eq. 3 / Eq. 1 (SI section 3 measures them at log-spaced times).  Layouts (int64):
 *   C[n_inst][R][L][n_tw][n_tm]  sum_i s_i(tm) s_i(tw) for tw <= tm <= tau, else 0
 *   q[n_inst][R/2][L][n_tm]      sum_i s_i^(2p)(tm) s_i^(2p+1)(tm)
 *   E[n_inst][R][L][n_tm]        VB: sum_{(ij) in E} J_ij s_i s_j;  SK: sum_{i<j} J_ij s_i s_j
 * (SK has L = 1.)  Entries whose time has not been reached are 0.  Each *_len is the capacity
 * in elements; a NULL pointer skips that array. */
int sg_read_results(sg_handle h, int64_t *C, size_t C_len, int64_t *q, size_t q_len,
                    int64_t *E, size_t E_len);

/* Window-averaged measurement (the estimator of the main text, "Extrapolation to large sizes
 * and large times": each point is the average of the measurements over a geometric window of
 * times, e.g. [t/2^(1/4), t]; SI section 1 lumps SK data in tritone windows the same way).
 * bounds[0] < bounds[1] < ... < bounds[n_bounds-1] (int64, host, >= 0, <= 2^32) cut time into
 * n_bounds-1 windows; window m holds the sweeps tau with bounds[m] <= tau < bounds[m+1].  Every
 * such tau is measured (after the snapshots due at tau) and its C, q, E are added into window m.
 * Must be called before sg_attach (the workspace size grows with the window count); otherwise
 * SG_ESTATE.  Invalid bounds: SG_EINVAL.  The point schedule (tw, tm) is unchanged. */
int sg_set_windows(sg_handle h, const int64_t *bounds, int32_t n_bounds);

/* Copy the window sums to the host (synchronises).  With n_bins = n_bounds - 1, layouts (int64):
 *   C[n_inst][R][L][n_tw][n_bins]  sum over measured tau in window m of C(tau, tw)
 *   q[n_inst][R/2][L][n_bins], E[n_inst][R][L][n_bins]  sums of q(tau), E(tau)
 *   n_meas[n_tw + 1][n_bins]  rows 0..n_tw-1: the number of taus summed into C for snapshot w
 *                             (tau >= tw[w], tau <= the current time); last row: for q and E
 * The window averages are C / n_meas.  SG_ESTATE if no windows were set. */
int sg_read_windows(sg_handle h, int64_t *C, int64_t *q, int64_t *E, int64_t *n_meas);

/* Measure now, at the current tau, against every snapshot taken so far (synchronises).
 * Defines: the same observables as sg_read_results (Eq. formula1, SI section 1), at one time.
 * C[n_inst][R][L][n_tw] (0 for snapshots not yet taken), q[n_inst][R/2][L], E[n_inst][R][L]. */
int sg_measure(sg_handle h, int64_t *C, size_t C_len, int64_t *q, size_t q_len, int64_t *E,
               size_t E_len);

/* Current spins in the caller's vertex order (synchronises).  The configuration {s_i} of
 * Eq. 1 / Eq. 3; the multispin word layout of SI section 2 for VB.
 *   VB: uint64[n_inst][R][n_g] concatenated over graphs, bit k = 1 iff s = -1 in lane k (bits
 *       >= n_lanes are 0 for SG_VB_PLAIN);  SK: int8[R][n] of +-1.
 * bytes must equal the exact size. */
int sg_get_spins(sg_handle h, void *host_dst, size_t bytes);

/* The acceptance threshold tables in use: VB uint32[n_inst][R][SG_VB_MAX_DEGREE+1] (entry m),
 * SK uint32[R][n] (entry k).  Entry 0 is 2^32-1.  Defines: the Metropolis acceptance
 * min(1, exp(-dE/T)) (Methods) as integer thresholds on a 32-bit random number. */
int sg_get_thresholds(sg_handle h, uint32_t *dst, size_t len);

/* VB: the colour class of every vertex of graph `graph` of the handle (int32[n], original
 * vertex labels) and the number of classes; a sweep updates class 0, 1, ... in turn.  Available
 * from creation (no device needed).  SG_EINVAL for an SK handle, a bad graph index or len < n.
 * Defines: the update order, one independent set at a time (the bipartite half-updates of SI
 * section 3, generalised by a greedy colouring and one recolouring pass). */
int sg_vb_colouring(sg_handle h, int32_t graph, int32_t *colour, size_t len, int32_t *n_colours);

/* Checkpoint: the full dynamic state (tau, spins, snapshots, counts) as an opaque host blob.
 * sg_state_bytes gives its size; sg_load_state restores it into an attached handle created
 * from the same instance.  Library service (long runs in pieces, as the paper's campaign of
 * Table 1 needed); the paper describes no checkpoint format. */
int sg_state_bytes(sg_handle h, size_t *bytes);
int sg_save_state(sg_handle h, void *host_dst, size_t bytes);
int sg_load_state(sg_handle h, const void *host_src, size_t bytes);

/* Release the handle (the workspace and stream stay the caller's).  Library service. */
int sg_destroy(sg_handle h);

/* Number of kernel launches the handle has queued since creation (for launch accounting).
 * Library service; no counterpart in the paper. */
int sg_launch_count(sg_handle h, int64_t *count);

/* Bytes the handle has copied host -> device (the instance image at attach, a loaded checkpoint)
 * and device -> host (results, spins, checkpoints) since creation (for transfer accounting).
 * Library service; no counterpart in the paper. */
int sg_transfer_bytes(sg_handle h, int64_t *h2d, int64_t *d2h);

/* The operations of one blocked SK sweep (blocks of 64 .. 512 spins, the launch-per-block
 * form) for n spins, in the order the library issues them, 6 int32 each: {op, stream, block,
 * skip0, skip1, event}.  op 0: the K* table; 1: the in-block kernel of block `block`; 2: the
 * update of every field row by that block; 3: the update of every row tile outside
 * [skip0, skip1); 4: record event `event` on `stream`; 5: make `stream` wait for it.  Stream 0
 * is the handle's stream, 1 its side stream; events 0 and 1 are "in-block done" (block parity),
 * 2 and 3 "side done".  *n_ops receives the number of operations; ops may be NULL with cap 0 to
 * query it; a smaller cap returns SG_EINVAL.  Needs no device.  Library service (host-side
 * checking of the launch schedule); no counterpart in the paper, whose SK sweep (SI section 1)
 * is sequential. */
int sg_sk_blocked_schedule(int32_t n, int32_t block, int32_t *ops, int32_t cap, int32_t *n_ops);

/* SK local fields h[r][i] = sum_j J_ij s[r][j] computed on the tensor cores without allocating
 * any device memory.  The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory where they need the fields -- a host application that fixes the
 * library's memory budget, or a plugin whose process owns every device allocation.
 *   J  device int8[n*n], row-major, +-1 off the diagonal, 0 on it, symmetric (not checked here)
 *   s  device int8[n_replicas*n], spins +-1, replica-major
 *   h  device int32[n_replicas*n], output, replica-major
 *   n  2..2048;  n_replicas a multiple of 16 in 16..128;  cuda_stream a cudaStream_t (or NULL)
 * The tensor-core operand images live in one static device array of about 5.3 MiB inside the
 * library (held by every GPU that loads it until the process exits); larger sizes return
 * SG_EINVAL.  J, s and h must be device memory of the current device.  The first call on a
 * device looks up that array's device address.  Every call reuses the array and clears what must
 * start at zero, so calls that overlap on the GPU (different streams or host threads) race with
 * each other: serialise them.  The call is queued on cuda_stream, synchronises that stream and
 * returns after its work completed; errors are reported like every other call (status code,
 * sg_last_error). */
int sg_sk_fields_noalloc(const int8_t *J, const int8_t *s, int32_t n, int32_t n_replicas,
                         int32_t *h, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
