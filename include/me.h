/*
 * me.h -- C ABI of the B300 matrix-element library (libme_b300.so).
 *
 * Evaluates tree-level matrix elements |M|^2 for batches of phase-space points on one
 * GPU, one event per CUDA thread.  This is the multi-event interface of the paper
 * (Section 3: random numbers, momenta and matrix elements produced in batches of up to
 * several thousand events and handed to an accelerated backend; Fig. 1c), and the
 * quantity computed is the one the paper offloads (abstract, Section 2): for each event
 *
 *     me = (1/IDEN) sum_{helicities h} sum_{colours} |M(p, h, colours)|^2 ,
 *
 * built from HELAS-style external wavefunctions, FFV / VVV / VVVV vertex currents for
 * every Feynman diagram, the helicity sum and the colour sum J^dagger C J over
 * colour-flow amplitudes J.  IDEN averages over initial spins and colours and divides
 * by n! for every set of n identical final particles (gluons, or the light quarks of
 * "u u > t t~ u u" and "u~ u~ > t t~ u~ u~").
 *
 * Processes (particle order of the string):
 *   "e+ e- > mu+ mu-"      2 diagrams (photon, Z),   16 helicities,   1 colour flow
 *   "g g > t t~"           3 diagrams,              16 helicities,   2 colour flows
 *   "g g > t t~ g"         16 diagrams,             32 helicities,   6
 *   "g g > t t~ g g"       123 diagrams,            64 helicities,  24
 *   "g g > t t~ g g g"     1240 diagrams,          128 helicities, 120
 *   "u u~ > t t~"          1 diagram,               16 helicities,   2 (a light quark
 *   "u~ u > t t~"          from either beam: the quark-initiated channel of p p -> t t~)
 *   "u u~ > t t~ g"        5 diagrams,              32 helicities,   4 (the one-jet quark
 *   "u~ u > t t~ g"        channels of p p -> t t~ + jet, either beam order; with
 *   "u g > t t~ u"         "g g > t t~ g" every channel of p p -> t t~ + 1 jet for one
 *   "g u > t t~ u"         massless light flavour.  Colour flows over the colours of
 *   "u~ g > t t~ u~"       the light line's row end B (incoming antiquark or outgoing
 *   "g u~ > t t~ u~"       quark), column end K, top t, antitop tb and gluon a:
 *                          T^a_{B tb} d_{t K}, T^a_{t K} d_{B tb}, T^a_{B K} d_{t tb},
 *                          T^a_{t tb} d_{B K})
 *   "u u~ > t t~ g g"      36 diagrams,             64 helicities,  13 (the two-jet
 *   "u~ u > t t~ g g"      channels of p p -> t t~ + 2 jets with one light-quark line,
 *   "u g > t t~ u g"       either beam order; with "g g > t t~ g g" all of them but
 *   "g u > t t~ u g"       the four-quark channels.  Flows over B, K, t, tb and the
 *   "u~ g > t t~ u~ g"     gluons a, b (a the lower particle index):
 *   "g u~ > t t~ u~ g"     (T^a T^b)_{B tb} d_{t K}, (T^b T^a)_{B tb} d_{t K},
 *   "g g > t t~ u u~"      T^a_{B tb} T^b_{t K}, T^b_{B tb} T^a_{t K}, d_{B tb} (T^a T^b)_{t K},
 *                          d_{B tb} (T^b T^a)_{t K}, the same six with (B K, t tb) in
 *                          place of (B tb, t K), and d^{ab} d_{B tb} d_{t K})
 *   "u u~ > t t~ d d~"     7 diagrams,              64 helicities,   6 (the four-quark
 *   "u~ u > t t~ d d~"     channels of p p -> t t~ + 2 jets with two light flavours:
 *   "u d > t t~ u d"       three fermion lines, u, d and top.  Flows over each line's
 *   "u d~ > t t~ u d~"     row end B (incoming antiquark or outgoing quark) and column
 *   "u~ d~ > t t~ u~ d~"   end K: d_{Bu K_s0} d_{Bd K_s1} d_{t K_s2} for the permutations
 *                          s of (Ku, Kd, tb) in lexicographic order)
 *   "u u > t t~ u u"       14 diagrams,             64 helicities,   6 (the four-quark
 *   "u~ u~ > t t~ u~ u~"   channels with one light flavour: both pairings of the light
 *   "u u~ > t t~ u u~"     quarks into lines, the second with the sign -1 of exchanging
 *   "u~ u > t t~ u u~"     identical fermions; the same six flows, the first pairing's
 *                          lines taken as the u and d lines above)
 *
 * Conventions:
 *   momenta   (E, px, py, pz) in GeV, FP64, array-of-structures [nevt][npar][4];
 *   helicity  index h in [0, 2^npar): particle i has helicity +1 if bit (npar-1-i) of h
 *             is set, else -1 (the physical helicity of that particle);
 *   colour    flow index = lexicographic rank of the gluon permutation s of the string
 *             (T^{a_s1} ... T^{a_sn})_{i_t j_tbar} (gluons named by particle index) for
 *             the gluon processes; the flows listed above for the quark channels;
 *   selection sel_hel = first kept helicity whose running sum of |M_h|^2 exceeds
 *             rnd_hel * total; sel_col = first flow whose running sum of
 *             w_i = sum_h |J_{h,i}|^2 exceeds rnd_col * sum_i w_i; both 0-based; an event
 *             whose total is 0 selects 0.
 *
 * Ownership: the caller owns every array passed to me_compute (device memory, for
 * example torch CUDA tensors).  The library owns the handle and what it keeps on the
 * device (helicity list, per-stream workspace).
 *
 * Errors: every call returns 0 on success or a negative status; me_last_error gives
 * the message.  Non-finite momenta produce NaN in me for that event only.
 *
 * Device-side timeouts: the mixed-precision kernel waits for its tensor-core work with
 * a bounded spin.  If a wait runs out (it never should), the kernel records it in a
 * flag of the handle, sets the matrix element of every event of that main pass to NaN
 * (its selections to 0; the FP64 rescue pass that follows may still fill in the events
 * it re-evaluates), and exits cleanly, so the CUDA context stays usable.  The host learns
 * of it asynchronously: me_sync_status reports it; otherwise the next me_compute or
 * me_compute_noalloc on the handle returns ME_ERR_TIMEOUT instead of computing, and
 * me_compute_host reports it for its own call.  Reporting clears the flag.
 */
#ifndef ME_B300_H
#define ME_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ME_OK 0
#define ME_ERR_ARG (-1)        /* null pointer, nevt < 0, unknown process, host pointer */
#define ME_ERR_MODE (-2)       /* precision mode not available for this process */
#define ME_ERR_NOMEM (-3)      /* device allocation failed */
#define ME_ERR_CUDA (-4)       /* a CUDA runtime call or kernel launch failed */
#define ME_ERR_TIMEOUT (-5)    /* a bounded device-side wait gave up */

#define ME_PREC_FP64 0   /* everything in FP64 */
#define ME_PREC_FP32 1   /* FP32 amplitudes and colour sum; FP64 inputs, denominators, helicity sum */
#define ME_PREC_MIXED 2  /* FP32 amplitudes, colour sum on tensor cores (split BF16/FP16 operands,
                            FP32 accumulation); FP64 inputs, denominators, helicity sum */
#define ME_PREC_DFLOAT 3 /* FP64-emulating amplitudes and colour sum in double-float arithmetic
                            (hi + lo FP32 pairs, about 48 significant bits, FP32 exponent range)
                            on the FP32 pipe; FP64 inputs, error-free invariants and helicity sum
                            as in FP64 mode.  Built for "g g > t t~", "g g > t t~ g" and the
                            six one-jet quark channels; ME_ERR_MODE elsewhere */

typedef struct me_handle me_handle;

/* Standard-model input parameters.  The weak mixing angle follows from (alpha, G_F,
 * mZ): mW^2 = mZ^2/2 + sqrt(mZ^4/4 - pi alpha mZ^2/(sqrt2 G_F)), sw^2 = 1 - mW^2/mZ^2. */
typedef struct {
  double mZ, wZ;            /* Z mass and width [GeV] */
  double mt, wt;            /* top mass and width [GeV] */
  double aEWM1;             /* 1/alpha_EM */
  double Gf;                /* Fermi constant [GeV^-2] */
  double alphas_default;    /* alpha_s when me_compute gets alphas == NULL */
  int precision;            /* ME_PREC_* (ME_ERR_MODE from me_init where a mode is not built) */
  int zero_width_tchan;     /* 1: no width in t-channel propagators (those that separate
                               the two incoming particles); Section 3, Tables 1-2 */
  double rescue_kappa;      /* FP32 and mixed modes: an event whose conditioning
                               kappa = max over gluon propagators of (sum of energies)^2/|K^2|
                               exceeds this is re-evaluated in FP64 (0 = never); nearly
                               collinear gluons make FP32 amplitudes lose digits */
} me_sm_params;

/* Fill p with the defaults: mZ 91.188, wZ 2.4414, mt 173, wt 1.4915, 1/alpha 132.5,
 * G_F 1.16639e-5, alpha_s 0.118, FP64, widths everywhere, rescue_kappa 2000. */
void me_default_params(me_sm_params* p);

/* Create a handle for one process on the current CUDA device.  Runs the helicity
 * filter: a helicity is kept when |M_h|^2 is not exactly zero (FP64) on any of 1024
 * fixed RAMBO events at sqrt(s) = 1500 GeV.  *out receives the handle (NULL on error).
 * Environment, read here: ME_B300_CONFIG selects the launch configuration (as
 * me_set_config); ME_B300_MAX_BLOCKS caps the blocks of the persistent grid, which
 * otherwise holds every block that fits on the device at once (for tests).
 * Errors: ME_ERR_ARG (null pointer, unknown process, invalid parameter),
 * ME_ERR_MODE, ME_ERR_NOMEM, ME_ERR_CUDA. */
int me_init(const char* process, const me_sm_params* p, me_handle** out);

/* Evaluate nevt events, asynchronously on cuda_stream (a cudaStream_t, NULL = legacy
 * default stream); results are ready when the stream reaches this point.
 *   momenta  device, FP64 [nevt][npar][4], 16-byte aligned
 *   alphas   device, FP64 [nevt], or NULL for alphas_default
 *   rnd_hel  device, FP64 [nevt] in (0,1), or NULL (then sel_hel is not written)
 *   rnd_col  device, FP64 [nevt] in (0,1), or NULL (then sel_col is not written)
 *   me       device, FP64 [nevt]                      (output, required)
 *   sel_hel  device, int32 [nevt] or NULL             (output)
 *   sel_col  device, int32 [nevt] or NULL             (output)
 * nevt == 0 is a no-op.  The handle keeps one workspace per stream (grown on demand,
 * stream-ordered); before capturing calls on a stream into a CUDA graph, size that
 * stream's workspace for the largest call with me_reserve (a later call that needs more
 * would move the workspace under the graph).  Calls on different streams may run
 * concurrently.
 * Errors: ME_ERR_ARG (null handle/momenta/me, nevt < 0, a host pointer, misaligned
 * momenta), ME_ERR_NOMEM, ME_ERR_CUDA, ME_ERR_TIMEOUT. */
int me_compute(me_handle* h, int64_t nevt, const double* momenta, const double* alphas,
               const double* rnd_hel, const double* rnd_col, double* me, int32_t* sel_hel,
               int32_t* sel_col, void* cuda_stream);

/* Same computation with HOST buffers: copies inputs to the device, computes, copies the
 * outputs back, and synchronises the stream before returning (end-to-end path).  The
 * host buffers should be pinned for full copy bandwidth.  Same argument meanings and
 * errors as me_compute, with host instead of device pointers. */
int me_compute_host(me_handle* h, int64_t nevt, const double* momenta, const double* alphas,
                    const double* rnd_hel, const double* rnd_col, double* me, int32_t* sel_hel,
                    int32_t* sel_col, void* cuda_stream);

/* The computation of me_compute with no device allocation on its path: no cudaMalloc,
 * cudaMallocAsync, cudaFree or allocating library routine.  It is meant for callers
 * that cannot let the library allocate -- a host framework that owns all device memory
 * through its own pool and forbids direct driver allocations, or a caller under a hard
 * memory cap or latency budget, where an allocation can fail or stall.  The paper has
 * no counterpart: it is an interface for such hosts.
 * The kernels' scratch (helicity running sums, slot buffer, momentum table, colour
 * weights) is one fixed 32 MiB device array inside the library, held on every GPU that
 * loads the library until the process exits.  A batch that needs more scratch than that
 * is rejected with ME_ERR_ARG and a message giving the exact largest batch that fits
 * (for "g g > t t~ g g" in FP64 about 9000 events per call).  The first call on a device,
 * and the first after the device's CUDA context was replaced (a device reset), looks up
 * the array's device address; make it before any stream capture.  Every call uses the
 * same array and leaves its contents behind: calls whose work overlaps on the GPU (other
 * streams, other handles) race on it, so the caller must serialise them.  Arguments,
 * outputs and the other errors are those of me_compute. */
int me_compute_noalloc(me_handle* h, int64_t nevt, const double* momenta, const double* alphas,
                       const double* rnd_hel, const double* rnd_col, double* me, int32_t* sel_hel,
                       int32_t* sel_col, void* cuda_stream);

/* Per-event subprocess dispatch.  A hadronic process is a sum of channels (for
 * p p -> t t~: g g -> t t~, u u~ -> t t~ and u~ u -> t t~, each light flavour having the
 * same matrix element), and an event generator produces the events of all channels in one
 * batch; the paper's outlook (Section 5) names this multi-subprocess case.  Event e of
 * the batch belongs to channel channel[e] and is evaluated by handle hs[channel[e]]:
 *   hs       host array of nchan (1 to 32) handles, all with the same number of
 *            particles, each in FP64 or FP32 (ME_ERR_MODE otherwise)
 *   channel  device, int32 [nevt]; an index outside [0, nchan) gives that event NaN in
 *            me and selections 0
 * and the other arguments as in me_compute (momenta in the particle order of the event's
 * channel).  Each event's results are those of me_compute with its channel's handle.
 * The partition by channel happens on the device; the call does not wait for it.  At
 * most 2^30 events per call.  Uses the first handle's workspace on cuda_stream for the
 * partition and each handle's own workspace for its channel.
 * Errors: ME_ERR_ARG (null or mismatched handles, nevt < 0, host pointers, misaligned
 * momenta), ME_ERR_MODE, ME_ERR_NOMEM, ME_ERR_CUDA, ME_ERR_TIMEOUT; messages on hs[0]. */
int me_compute_channels(me_handle* const* hs, int nchan, int64_t nevt, const int32_t* channel,
                        const double* momenta, const double* alphas, const double* rnd_hel,
                        const double* rnd_col, double* me, int32_t* sel_hel, int32_t* sel_col,
                        void* cuda_stream);

/* GPU-assisted batch unweighting (Section 3, Table 2): with the whole batch's largest
 * weight known before any decision, hit-or-miss needs no provisional storage.
 *   me       device, FP64 [nevt]  matrix elements (e.g. from me_compute)
 *   wgt      device, FP64 [nevt]  the rest of each event weight (Jacobian x PDFs ...)
 *   rnd      device, FP64 [nevt]  uniform numbers in [0,1); required when accept or
 *                                 n_accept is given
 *   w        device, FP64 [nevt]  output w_i = me_i * wgt_i, or NULL
 *   accept   device, uint8 [nevt] output 1 when w_i > rnd_i * w_max, else 0; or NULL
 *   w_max    device, one FP64     output: the largest valid weight (finite, >= 0), or 0
 *                                 when there is none; 8-byte aligned
 *   n_accept device, one int64    output: number of accepted events, or NULL
 * A weight that is NaN, infinite or negative never sets w_max and is never accepted.
 * Asynchronous on cuda_stream; nevt == 0 is a no-op that leaves the outputs untouched.
 * Errors: ME_ERR_ARG (null handle or required pointer, nevt < 0, a host pointer,
 * misaligned scalar), ME_ERR_CUDA. */
int me_unweight(me_handle* h, int64_t nevt, const double* me, const double* wgt, const double* rnd,
                double* w, uint8_t* accept, double* w_max, int64_t* n_accept, void* cuda_stream);

/* me_compute and me_unweight in one call: the event weight w_i = me_i * wgt_i and the
 * batch maximum are formed in the epilogue of the matrix-element kernel (the step that
 * writes me and the selections), the reduction the paper places beside the event
 * selection (Section 3, Table 2); then one pass decides accept_i = w_i > rnd_i * w_max.
 * Arguments as in me_compute, then:
 *   wgt, rnd     device, FP64 [nevt]   as in me_unweight (rnd needed for accept/n_accept)
 *   w, accept    device outputs as in me_unweight, or NULL
 *   w_max        device, one FP64, 8-byte aligned (output, required)
 *   n_accept     device, one int64, or NULL
 * The outputs equal those of me_compute followed by me_unweight on its results, bit for
 * bit.  In the FP32 and mixed modes an event re-evaluated by the FP64 rescue pass enters
 * w and w_max with its FP64 value only.  Errors: those of me_compute and me_unweight;
 * ME_ERR_MODE for a launch configuration with two events per thread. */
int me_compute_unweight(me_handle* h, int64_t nevt, const double* momenta, const double* alphas,
                        const double* rnd_hel, const double* rnd_col, const double* wgt, const double* rnd,
                        double* me, int32_t* sel_hel, int32_t* sel_col, double* w, uint8_t* accept,
                        double* w_max, int64_t* n_accept, void* cuda_stream);

/* Synthetic inputs generated on the device, for the standalone multi-event testbed
 * (Section 2, Fig. 1b): a batch of test events is made and evaluated without a host
 * round trip.  The numbers are those of the counter-based definition (Philox4x32-10,
 * Salmon et al. SC'11): every uniform is a function of (seed, event index, stream,
 * draw), key = (seed mod 2^32, seed div 2^32), counter = (event mod 2^32,
 * event div 2^32, draw div 2, stream), draw j from output words (x0, x1) for even j and
 * (x2, x3) for odd j, u = (((hi << 32 | lo) >> 12) + 1/2) 2^-52 in (0, 1); they do not
 * depend on how a workload is split into batches.
 *
 * me_rambo: RAMBO momenta (Kleiss, Stirling, Ellis 1986) for the handle's process at
 * sqrt_s, events first_event .. first_event + nevt - 1, from stream 0 (4 draws per
 * final-state particle); beams along +z and -z; massive final states (the top mass of
 * the handle's parameters) by one Newton-rescaled factor on all three-momenta.
 *   momenta  device, FP64 [nevt][npar][4] (output, (E, px, py, pz))
 * An event whose rescaling does not converge in 50 steps gets NaN momenta.
 * Errors: ME_ERR_ARG (null handle, nevt < 0, host pointer, sqrt_s not above the sum of
 * the final masses), ME_ERR_CUDA. */
int me_rambo(me_handle* h, int64_t nevt, uint64_t seed, uint64_t first_event, double sqrt_s, double* momenta,
             void* cuda_stream);

/* me_uniforms: out[i] = offset + scale * u(seed, first_event + i, stream_id, draw 0),
 * device FP64 [nevt].  Streams used by the benchmarks: 1 alpha_s (offset 0.10, scale
 * 0.03), 2 rnd_hel, 3 rnd_col (offset 0, scale 1).  Errors: ME_ERR_ARG (nevt < 0,
 * stream_id < 0, host pointer; message in me_last_error(NULL)), ME_ERR_CUDA. */
int me_uniforms(int64_t nevt, uint64_t seed, uint64_t first_event, int stream_id, double offset, double scale,
                double* out, void* cuda_stream);

/* Process shape: external particles, helicity combinations, helicities kept by the
 * filter, colour flows, Feynman diagrams.  Any output pointer may be NULL. */
int me_info(const me_handle* h, int* npar, int* ncomb, int* ngood, int* ncol, int* ndiag);

/* The helicity indices kept by the filter, ascending; list must hold ncomb entries. */
int me_good_helicities(const me_handle* h, int32_t* list);

/* Work per event for the roofline: real floating-point operations of one helicity's
 * amplitudes and of one helicity's colour sum, as counted by the code generator. */
int me_flops(const me_handle* h, int64_t* flops_amp_per_hel, int64_t* flops_col_per_hel);

/* Plan of a me_compute call of nevt events: the number of kernel launches it makes
 * and the bytes of stream workspace it needs (with both selection outputs requested).
 * Either output pointer may be NULL. */
int me_plan(const me_handle* h, int64_t nevt, int64_t* launches, int64_t* workspace_bytes);

/* Grow the handle's workspace on cuda_stream to what a me_compute call of nevt events
 * with both selection outputs needs under the current configuration, so that calls up
 * to that size on that stream allocate nothing (stream-ordered allocation on
 * cuda_stream).  Errors: ME_ERR_ARG (null handle, nevt < 0), ME_ERR_NOMEM, ME_ERR_CUDA. */
int me_reserve(me_handle* h, int64_t nevt, void* cuda_stream);

/* Launch geometry of the main pass of a me_compute call of nevt events: blocks of the
 * persistent grid, threads per block, resident blocks per SM of the kernel, SMs of the
 * handle's device.  Any output pointer may be NULL.  Errors: ME_ERR_ARG. */
int me_launch_shape(const me_handle* h, int64_t nevt, int* grid, int* block, int* blocks_per_sm, int* nsm);

/* Wait for cuda_stream, then report whether a device-side wait of an earlier call on
 * this handle ran out (see "Device-side timeouts" above): ME_OK, or ME_ERR_TIMEOUT
 * (the flag is then cleared).  Errors: ME_ERR_ARG (null handle), ME_ERR_CUDA. */
int me_sync_status(me_handle* h, void* cuda_stream);

/* Testing hook for the timeout path: the number of polls the mixed kernel's wait for
 * its tensor-core work makes before it gives up, for later calls on this handle.
 * polls < 0 restores the default (2^22 polls); 0 makes the wait give up at once, so
 * that a test can drive the timeout path without any fault.  The kernel's final wait,
 * which keeps its tensor memory allocated until every issued MMA has completed, always
 * keeps the default limit.  Errors: ME_ERR_ARG (null handle). */
int me_set_wait_limit(me_handle* h, int64_t polls);

/* Select the kernel launch configuration (register budget, block size, placement of
 * per-thread arrays) used by later me_compute calls; 0 is the default.  Returns the
 * number of configurations available for the handle's precision when config < 0.
 * Errors: ME_ERR_ARG for an unknown configuration. */
int me_set_config(me_handle* h, int config);

/* Message of the last failing call on this handle (or of the last failing me_init when
 * h is NULL).  Never NULL; "" when there was no error. */
const char* me_last_error(const me_handle* h);

/* Release the handle and its device memory (synchronises the device). */
void me_free(me_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* ME_B300_H */
