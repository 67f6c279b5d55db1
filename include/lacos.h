/*
 * lacos.h -- C ABI of the GB300 L.A.Cosmic detect-and-clean library.
 *
 * The operation is the cosmic-ray detection and cleaning iteration of
 * L.A.Cosmic (van Dokkum 2001) as ported by dfcosmic (arXiv 2602.17938,
 * Methods / "Algorithm", steps 1-7, and "Main parameters"):
 *   1. Laplacian detection: the image is block-replicated 2x, convolved with
 *      the 3x3 Laplacian, clipped at zero and block-averaged back (L+);
 *   2. noise model N = sqrt(max(gain*med5(I), 1e-4) + readnoise^2) / gain;
 *   3. significance S = L+ / (2N), and S' = S - med5(S);
 *   4. candidates: S' > sigclip;
 *   5. compact objects rejected: S'/F > objlim with the fine-structure image
 *      F = max((med3(I) - med7(med3(I))) / N, 0.01);
 *   6. neighbours included by two 3x3 growth steps re-tested against sigclip
 *      and sigfrac*sigclip; saturated pixels (input >= satlevel) never flag;
 *   7. flagged pixels replaced by the median of the unflagged input pixels
 *      of their 5x5 window (lower median for even counts; widened to 7x7,
 *      9x9, ... when none is unflagged);
 * repeated up to niter times, stopping early once an iteration flags no new
 * pixel.  Medians are true (non-separable) K x K medians with clamp-to-edge
 * borders.  Arithmetic is IEEE float32 (no FMA contraction), and results are
 * bit-identical to a plain float32 CPU implementation of the same steps.
 *
 * Layout: every image is row-major, ny rows of nx pixels, row stride nx,
 * contiguous, in device memory (except where a call says "host").
 *
 * Ownership: the caller owns frames and outputs and keeps them alive and
 * untouched from submit until poll reports completion.  The library owns
 * its scratch (5 bits per pixel, 6 with satgrow > 0, plus 512 KiB and 3
 * bytes per 32x32 tile per frame, and 1.5 MiB for a frame whose gain is
 * estimated; lacos_request_bytes gives the figure), charged against the
 * context's HBM budget.
 *
 * Errors: every call returns an int status; 0 is success.  Negative values
 * are the LACOS_E* codes below; lacos_poll also returns LACOS_PENDING (1).
 * Calls are thread-safe on one context.
 */
#ifndef LACOS_H
#define LACOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lacos_ctx lacos_ctx; /* opaque, library-owned */
typedef struct CUstream_st *lacos_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum { LACOS_F32 = 0, LACOS_U16 = 1 } lacos_dtype;

enum {
  LACOS_OK = 0,
  LACOS_PENDING = 1,
  LACOS_EINVAL = -1,          /* bad pointer, size or parameter */
  LACOS_EAGAIN = -2,          /* no free slot or budget right now: retry later */
  LACOS_ENOMEM = -3,          /* the request can never fit the context's budget */
  LACOS_ECUDA = -4,           /* a CUDA call failed; see lacos_last_cuda_error */
  LACOS_ENONFINITE = -5,      /* the input held NaN or Inf: outputs undefined */
  LACOS_ETIMEOUT = -6,        /* a bounded device wait gave up */
  LACOS_EUNKNOWN_TICKET = -7, /* poll on a ticket that is not in flight */
  LACOS_ENOGAIN = -8          /* an estimated gain was undefined at some iteration (no pixel
                                 pair left, or all their differences equal); that iteration
                                 used gain 1 */
};

#define LACOS_MAX_NITER 256

/* Parameters of one frame (dfcosmic "Main parameters" plus gain, readnoise).
 * gain > 0 [e-/ADU], or 0 to estimate it at every iteration ("Main
 * parameters": a gain that is not supplied is estimated per iteration; the
 * paper gives no formula, so this library's reading is photon transfer on
 * adjacent pixel pairs).  At iteration k the pairs (columns 2m, 2m+1) whose
 * pixels are both unflagged so far and unsaturated give d = a - b; d is
 * clipped at 3 population standard deviations from its mean (exactly, in
 * integers; at most 5 rounds, stopping when a round keeps every pair), and g
 * solves V g^2 - A g - 2 n rn^2 = 0 for the n remaining pairs, V the sum of
 * squared deviations of d and A the sum of a + b, evaluated in double and
 * rounded to float.  Only uint16 frames (float32 frames with gain 0 are
 * LACOS_EINVAL).  readnoise >= 0 [e-]; satlevel [ADU], <= 0 disables the
 * saturation guard; sigclip, sigfrac, objlim > 0; 0 <= niter <= 256.
 * fine_norm: 1 divides the fine-structure image by N (default reading),
 * 0 uses max(med3 - med7, 0.01) unnormalised.
 * satgrow: 0..4, saturated-star protection: the pixels within this many
 * pixels (Chebyshev distance) of a saturated input pixel are treated as
 * saturated too (never flagged, never replaced); 0 protects only the
 * saturated pixels themselves.
 * sepmed: 0 (the method), or 1 for the comparison mode that takes both 5x5
 * detection medians (noise model, large-structure removal) separably: the
 * median of the five row medians, as faster implementations do. */
typedef struct {
  float gain, readnoise, satlevel, sigclip, sigfrac, objlim;
  int niter;
  int fine_norm;
  int satgrow;
  int sepmed;
} lacos_params;

typedef struct {
  int status;            /* LACOS_OK or LACOS_ENONFINITE / LACOS_ETIMEOUT / LACOS_ENOGAIN */
  int iters_run;         /* iterations executed (early stop included) */
  long long n_flagged;   /* pixels in the final cosmic-ray mask */
  double latency_ms;     /* submit-to-completion on the device (event time) */
  float gain;            /* the gain of the last iteration run: the supplied one, or the
                            estimate when gain = 0 (0 if no iteration ran); 0 for the
                            aggregate of a batch of several frames */
} lacos_result;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * library-owned scratch (0 = 8 GiB); max_slots caps requests in flight
 * (0 = 64).  *out receives the context. */
int lacos_create(lacos_ctx **out, int device, size_t hbm_budget_bytes, int max_slots);

/* Queue the detect-and-clean of one frame on `stream` (work is ordered
 * after everything already queued on it; the outputs are complete when the
 * completion event recorded on `stream` fires).
 *   d_frame : ny*nx float32 (LACOS_F32) or uint16 (LACOS_U16) pixels [ADU]
 *   d_mask  : out, ny*nx uint8, 1 = cosmic ray (cumulative over iterations)
 *   d_clean : out, ny*nx float32 cleaned frame
 *   ticket  : out, identifies the request for lacos_poll
 * Requires 1 <= ny, nx and ny*nx < 2^31.  Returns LACOS_EAGAIN when no slot
 * or budget is free (nothing was queued). */
int lacos_submit(lacos_ctx *c, const void *d_frame, lacos_dtype dt, int ny, int nx,
                 const lacos_params *p, uint8_t *d_mask, float *d_clean,
                 lacos_stream stream, unsigned long long *ticket);

/* As lacos_submit, but the request runs on a stream of its own (one per
 * slot, created on first use), so requests submitted back to back overlap
 * on the device -- the continuous batching of the serving loop: a request is
 * admitted as soon as a slot and budget are free, whatever is still running.
 * The work is ordered after nothing the caller queued: the frame must
 * already be complete on the device when the call is made. */
int lacos_submit_async(lacos_ctx *c, const void *d_frame, lacos_dtype dt, int ny, int nx,
                       const lacos_params *p, uint8_t *d_mask, float *d_clean,
                       unsigned long long *ticket);

/* Host-to-host request: copies the host frame into device buffers the slot
 * owns (charged to the budget, reused across requests), runs the request,
 * and copies the mask and cleaned frame back into the host buffers, all on
 * the slot's own stream; lacos_poll/lacos_wait report completion once the
 * host outputs are written.  Requests submitted back to back use different
 * slots and streams, so one frame's upload, another's compute and a third's
 * download overlap (separate copy engines).  Frames of at least 8 x the
 * GPU's resident core CTAs in 32x64 tiles (about 10 Mpx on 152 SMs) run
 * their kernels in submission order, one such request at a time, so that
 * the copies overlap compute; smaller frames run concurrently, and several
 * more in flight raise their throughput.
 *   h_frame : in, ny*nx host pixels (LACOS_F32 float32 or LACOS_U16 uint16)
 *   h_mask  : out, ny*nx uint8 host mask
 *   h_clean : out, ny*nx float32 host cleaned frame
 * Host buffers should be page-locked (cudaHostAlloc or registered) for the
 * copies to overlap; the caller keeps them alive and leaves h_frame
 * unchanged until completion.  Errors as lacos_submit (LACOS_EAGAIN when no
 * slot or budget is free). */
int lacos_submit_host(lacos_ctx *c, const void *h_frame, lacos_dtype dt, int ny, int nx,
                      const lacos_params *p, uint8_t *h_mask, float *h_clean,
                      unsigned long long *ticket);

/* Non-blocking completion check.  Returns LACOS_PENDING while the request
 * runs; otherwise fills *res, releases the request's slot and returns
 * LACOS_OK (res->status carries LACOS_ENONFINITE/LACOS_ETIMEOUT if the device
 * reported one).  A ticket can be polled to completion once. */
int lacos_poll(lacos_ctx *c, unsigned long long ticket, lacos_result *res);

/* Block until the request completes, then behave as lacos_poll. */
int lacos_wait(lacos_ctx *c, unsigned long long ticket, lacos_result *res);

/* Batched form: n frames of any sizes and dtypes processed together, one
 * launch per iteration level over a shared tile work queue (and a CUDA
 * graph replayed when the same batch is submitted again with
 * reuse_graph != 0).  1 <= n <= 65535.  Arrays have n entries; params may
 * differ per frame (niter included).  One ticket covers the whole batch; its lacos_result
 * sums n_flagged and reports the largest iters_run; per-frame results go
 * to per_frame (host array of n, may be NULL) when the batch is polled. */
int lacos_submit_batch(lacos_ctx *c, int n, const void *const *d_frames, const int *dtypes,
                       const int *ny, const int *nx, const lacos_params *params,
                       uint8_t *const *d_masks, float *const *d_cleans, lacos_stream stream,
                       int reuse_graph, lacos_result *per_frame, unsigned long long *ticket);

/* Kernel-level profile of the most recent request completed on the context
 * (filled only while profiling is switched on with lacos_set_profiling; the
 * times come from CUDA events recorded between the request's launches on
 * its stream, so requests replayed from a CUDA graph are not profiled). */
typedef struct {
  int n_levels;                        /* iteration levels launched */
  float core_ms[LACOS_MAX_NITER];      /* per level: step 7 of the previous level, steps 1-5; when
                                          the gain is estimated, also that level's estimate (the
                                          pair histogram, its clipping rounds and the N table) */
  float grow_ms[LACOS_MAX_NITER];      /* per level: step 6 (growth, mask update) */
  float final_ms;                      /* cleaned frame (last step 7) and uint8 mask */
  long long px_iterations;             /* sum over frames of ny*nx*iters_run */
  long long n_sprime;                  /* pixels where S' = S - med5(S) was evaluated */
  long long n_fine;                    /* pixels where the fine-structure F was evaluated */
  long long n_replace;                 /* masked-median replacements inside core launches */
  long long n_replace_wide;            /* ... of which the 5x5 window was fully flagged */
  long long px_core;                   /* tile pixels the core kernel computed, all levels (a
                                          level recomputes only tiles whose inputs changed) */
  long long n_sprime_net;              /* ... of n_sprime, those that ran the med5 network (the
                                          others needed only the lo test, decided by rank) */
  long long n_fine_net;                /* ... of n_fine, those that ran the med7 network (float32
                                          frames; uint16 frames decide the objlim test by rank) */
} lacos_profile;

int lacos_set_profiling(lacos_ctx *c, int on);
int lacos_last_profile(lacos_ctx *c, lacos_profile *out);

/* Detect-and-clean of one frame without any device allocation.  The paper
 * has no counterpart: this serves callers that must not allocate device
 * memory while they run -- a pipeline that plans all GPU memory at start-up
 * and forbids cudaMalloc afterwards (an allocation can synchronise the
 * device and break the plan), or a plugin whose host application owns the
 * device allocator.  The scratch lives in a fixed array of
 * LACOS_STATIC_SCRATCH_BYTES inside this library's device image, held by
 * every GPU that loads the library until the process exits; frames whose
 * scratch (lacos_request_bytes(ny, nx, p)) exceeds it are rejected with
 * LACOS_ENOMEM: above about 106 Mpx with satgrow = 0 (five bit-planes;
 * 9576 x 6388 fits, 12000 x 12000 does not), above about 88 Mpx with
 * satgrow > 0 (a sixth plane holds the grown saturated set); an estimated
 * gain needs 1.5 MiB more for its histogram.  Arguments,
 * layout and results are those of lacos_submit (outputs written to the
 * caller's d_mask and d_clean), except res->latency_ms: the host time from
 * entry to return, since the call queues the work on `stream`, waits for it
 * and then fills *res (may be NULL).  The first
 * call on a device looks up the array's device address and the launch
 * geometry for that device (no allocation); make that first call before
 * any stream capture.  All calls share the one array and it keeps the last
 * call's contents (the call clears what must start at zero), so calls that
 * overlap on the GPU -- from several host threads or streams -- race and
 * must be serialised by the caller. */
#define LACOS_STATIC_SCRATCH_BYTES (64u << 20)
int lacos_run_static(const void *d_frame, lacos_dtype dt, int ny, int nx, const lacos_params *p,
                     uint8_t *d_mask, float *d_clean, lacos_stream stream, lacos_result *res);

/* Core-kernel variant of the context: the tile shape of the detection
 * kernel and the resident CTAs per SM its registers are bounded for.
 *   0..3: 32 x 64 tiles, 256 threads, 1..4 CTAs per SM (more CTAs hide more
 *         latency, fewer registers spill more; 3 is the default);
 *   4, 5: 64 x 64 tiles, 512 threads, 1 or 2 CTAs per SM;
 *   6, 7: 32 x 128 tiles, 512 threads, 1 or 2 CTAs per SM;
 *   8, 9: 32 x 32 tiles, 160 threads, 5 or 6 CTAs per SM.
 * Larger tiles recompute less of the halo (each tile evaluates its medians
 * up to 6 pixels beyond its edges) but hold more shared memory per CTA.
 * lacos_autotune runs the given frame `reps` times (after one warm-up) with
 * each variant, keeps the fastest, and reports each variant's mean device
 * time in variant_ms[LACOS_CORE_VARIANTS] (may be NULL).  Results do not
 * depend on the variant. */
#define LACOS_CORE_VARIANTS 10
int lacos_set_core_variant(lacos_ctx *c, int variant);
int lacos_get_core_variant(lacos_ctx *c, int *variant);
int lacos_autotune(lacos_ctx *c, const void *d_frame, lacos_dtype dt, int ny, int nx,
                   const lacos_params *p, uint8_t *d_mask, float *d_clean, lacos_stream stream,
                   int reps, int *best_variant, float *variant_ms);

/* Drain in-flight work, free all library memory and the context. */
int lacos_destroy(lacos_ctx *c);

/* Scratch bytes a frame of ny x nx needs with default parameters
 * (satgrow = 0); what the budget is charged for such a request. */
size_t lacos_scratch_bytes(int ny, int nx);

/* Scratch bytes a request for one ny x nx frame with parameters *p (NULL:
 * defaults) is charged against the budget; satgrow > 0 adds one bit-plane,
 * gain = 0 the 1.5 MiB histogram of the gain estimate.  0 for empty extents. */
size_t lacos_request_bytes(int ny, int nx, const lacos_params *p);

/* Last CUDA error code seen by the context (0 if none). */
int lacos_last_cuda_error(lacos_ctx *c);

/* Library version string, "lacos-gb300 <major>.<minor> (sm_103a)"; the number
 * changes with the ABI (0.2: lacos_result.gain, LACOS_ENOGAIN, gain = 0;
 * 0.3: lacos_request_bytes). */
const char *lacos_version(void);

/* Self-check of the division the uint16 path uses instead of IEEE division
 * (S = L+/(2N) from a table of 2N and its correctly rounded reciprocal,
 * with Markstein's correction; the float32 path divides directly).  For the
 * given gain and read noise it builds the 65536-entry table and compares,
 * bit for bit, the result with IEEE float32 division for every numerator a
 * uint16 frame's L+ can take (k/4, k = 0..524280) and every entry: 3.4e10
 * pairs on the current device, tens of milliseconds.  *mismatches receives
 * the number of differing pairs (0 means identical everywhere).
 * Errors: LACOS_EINVAL (null pointer, gain <= 0, negative or non-finite
 * values), LACOS_ECUDA.  Allocates and frees 8 bytes of device memory. */
int lacos_selftest_division(float gain, float readnoise, unsigned long long *mismatches);

#ifdef __cplusplus
}
#endif

#endif /* LACOS_H */
