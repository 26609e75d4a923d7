/*
 * dgf.h - C ABI of the fast guided filtering layer on sm_103a.
 *
 * The layer (Wu et al., "Fast End-to-End Trainable Guided Filter") maps a
 * low-resolution target p_l (the paper's O_l), a low-resolution guide I_l
 * and a high-resolution guide I_h, with window radius r and ridge eps, to
 * the high-resolution output O_h (Sec. 3.1-3.3):
 *
 *   mean_I, mean_p, var_I, cov_Ip over every (2r+1)^2 window of the
 *   low-resolution grid, clipped to the image and divided by the number of
 *   in-image pixels;  A = cov_Ip / (var_I + eps),  b = mean_p - A mean_I
 *   (Eq. 1);  Abar, bbar = box means of A and b;  Abar_h, bbar_h = bilinear
 *   upsampling to h x w with half-pixel centres (align_corners = False);
 *   O_h = Abar_h * I_h + bbar_h  (Eq. 2).
 *
 * dgf_backward returns the gradients of Algorithm 1 (with respect to p_l,
 * I_l and I_h, extended through the box mean of A and b).  With a guidance
 * transform F (Sec. 3.4: 1x1 conv, leaky ReLU, 1x1 conv) the guides become
 * G_h = F(I_h) and G_l = the f x f block mean of G_h (or F(I_l) with
 * dgf_options.guide_low), and the weight gradients are returned as well.
 * A guide whose channel count differs from the output's is replaced by its
 * channel mean (dgf_options.guide_channels, Sec. 4.2, DGF_b).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout:    every image tensor is NCHW, contiguous, planes back to back:
 *            element (n, c, y, x) of an N x C x H x W tensor is at
 *            ((n*C + c)*H + y)*W + x.
 * Memory:    every tensor pointer is DEVICE memory owned by the caller
 *            (dgf_host_step alone takes HOST tensors).  The library
 *            allocates no tensor memory; it uses the caller's workspace
 *            (dgf_workspace_size bytes, or dgf_workspace_size_opt for the
 *            _opt calls; 256-byte aligned) for its intermediates.
 * Precision: storage is FP32, BF16 or FP16 (dgf_dtype); every sum and every
 *            product is formed in FP32; stores round to nearest even.
 * Streams:   calls enqueue kernels on `stream` and return without waiting.
 *            A workspace may be reused by calls on the same stream; calls
 *            that overlap on the device need separate workspaces.  Calls
 *            that pass a guidance transform stage its 93 weights in the
 *            library's constant memory, so such calls must not overlap on
 *            the device (serialise them on one stream).
 * Errors:    arguments are validated on the host before anything is
 *            enqueued; a bad argument returns DGF_ERR_INVALID (or
 *            DGF_ERR_UNSUPPORTED / DGF_ERR_WORKSPACE) and enqueues nothing.
 *            A CUDA error at launch returns DGF_ERR_CUDA.  dgf_last_error()
 *            gives a message for the calling thread's last non-OK status.
 *            No entry point aborts, traps or prints.
 * Sizes:     1 <= h_l <= h and 1 <= w_l <= w; the scale is the size ratio,
 *            so non-integer ratios are accepted.  r >= 0, eps finite and
 *            at least FLT_MIN (the smallest normal float; 1/(var + eps) is
 *            taken with the hardware's approximate reciprocal), N >= 0,
 *            C >= 1 (C = 3 when a guidance transform is given).  N = 0 is a
 *            valid empty call.
 */
#ifndef DGF_H
#define DGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* dgf_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum { DGF_F32 = 0, DGF_BF16 = 1, DGF_F16 = 2 } dgf_dtype;

typedef enum {
    DGF_OK = 0,
    DGF_ERR_INVALID = 1,     /* bad pointer, size, radius, eps or dtype   */
    DGF_ERR_UNSUPPORTED = 2, /* valid but not implemented (e.g. C != 3 with a guide) */
    DGF_ERR_CUDA = 3,        /* a CUDA runtime call failed                */
    DGF_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out        */
    DGF_ERR_WORKSPACE = 5    /* workspace missing, misaligned or too small */
} dgf_status;

/*
 * Guidance transform F of Sec. 3.4 / Table 1 (1x1 convolutions, no
 * normalisation): hidden = w1 . x (no bias), leaky ReLU with `slope`,
 * G = w2 . lrelu(hidden) + b2, per pixel, C = 3 in and out.
 * w1: hidden x 3 row-major, w2: 3 x hidden row-major, b2: 3; all FP32
 * DEVICE pointers.  1 <= hidden <= 16.  A NULL dgf_guide* means F = identity.
 */
typedef struct {
    const float* w1;
    const float* w2;
    const float* b2;
    int hidden;
    float slope;
} dgf_guide;

/* One image of a batched call (per-image sizes, radius, eps; C channels).
 * coef: NULL, or C x h_l x w_l FP32 (Abar, bbar) pairs (8-byte aligned) the
 * forward writes the image's coefficients to (as dgf_options.coef), for a
 * batched backward that takes them (dgf_image_grad.coef). */
typedef struct {
    const void* p_l; /* C x h_l x w_l */
    const void* I_l; /* C x h_l x w_l */
    const void* I_h; /* C x h x w     */
    void* O_h;       /* C x h x w     */
    int C, h_l, w_l, h, w, r;
    float eps;
    void* coef;
} dgf_image;

/*
 * Bytes of workspace that dgf_forward and dgf_backward need for these sizes
 * (the larger of the two; FP32 Abar/bbar, their gradients, the window
 * statistics; when g != NULL also the low-res guide, weight-gradient
 * partials and F(I_h) in FP32, N x 3 x h x w, which the forward computes
 * once for the block mean and reads back for Eq. 2).  Returns 0 for invalid
 * sizes.  Pure host function.
 */
size_t dgf_workspace_size(int N, int C, int h_l, int w_l, int h, int w, int r,
                          dgf_dtype dt, const dgf_guide* g);

/*
 * Forward pass, Eq. 1-2 with the box mean of A and b (Sec. 3.2-3.3).
 * p_l, I_l: N x C x h_l x w_l; I_h, O_h: N x C x h x w; all of dtype dt.
 * With g != NULL, I_l is ignored (may be NULL): the low-resolution guide is
 * the f x f block mean of F(I_h), which requires h = f*h_l and w = f*w_l.
 */
dgf_status dgf_forward(const void* p_l, const void* I_l, const void* I_h, void* O_h,
                       int N, int C, int h_l, int w_l, int h, int w, int r, float eps,
                       dgf_dtype dt, const dgf_guide* g,
                       void* workspace, size_t ws_bytes, dgf_stream_t stream);

/*
 * Backward pass, Algorithm 1 extended through the box mean of A and b.
 * dO_h is the upstream gradient dL/dO_h (N x C x h x w, dtype dt).  Outputs
 * (each nullable = not wanted): dp_l, dI_l (N x C x h_l x w_l, dtype dt),
 * dI_h (N x C x h x w, dtype dt), and with g != NULL dW: 3*hidden + 3*hidden
 * + 3 FP32 values laid out [dw1 | dw2 | db2], OVERWRITTEN with the sum over
 * the batch.  With g != NULL, dI_l must be NULL (I_l is not an input).
 * Every statistic is recomputed from the inputs; nothing from the forward
 * call is needed.
 */
dgf_status dgf_backward(const void* dO_h, const void* p_l, const void* I_l, const void* I_h,
                        void* dp_l, void* dI_l, void* dI_h, float* dW,
                        int N, int C, int h_l, int w_l, int h, int w, int r, float eps,
                        dgf_dtype dt, const dgf_guide* g,
                        void* workspace, size_t ws_bytes, dgf_stream_t stream);

/* Workspace bytes for dgf_forward_batched on this list (0 if invalid). */
size_t dgf_workspace_size_batched(const dgf_image* imgs, int n, dgf_dtype dt);

/*
 * Forward pass of n images of different sizes, radii and scale factors
 * (same dtype, F = identity) in one persistent launch per stage, replayed
 * from a CUDA graph that the library builds once per (dtype, device) and
 * updates in place on later calls.  Each image is computed exactly as
 * dgf_forward computes it with the same tile configuration, so results are
 * bitwise identical to per-image calls.  n <= DGF_MAX_BATCH.
 * The image table is read on the host during the call; it need not outlive it.
 * The workspace (dgf_workspace_size_batched) holds each image's
 * coefficients and a tensor map per image for the TMA-staged high-res
 * strips (16-byte vectors), copied into it on `stream` from host memory
 * before the graph runs (under stream capture the strips read with plain
 * loads instead: the same bits).
 */
#define DGF_MAX_BATCH 128
dgf_status dgf_forward_batched(const dgf_image* imgs, int n, dgf_dtype dt,
                               void* workspace, size_t ws_bytes, dgf_stream_t stream);

/* Message for the calling thread's last non-OK status ("" if none). */
const char* dgf_last_error(void);

/*
 * Optional per-kernel timing with CUDA events recorded on the launch stream
 * around every kernel the library enqueues (for benchmarks).  While enabled,
 * each call synchronises its stream before returning, to read the events.
 * dgf_profile_read fills up to `cap` entries of names/milliseconds/launches
 * accumulated since the last reset and returns the number of kernel kinds.
 */
void dgf_profile_enable(int on);
void dgf_profile_reset(void);
int dgf_profile_read(const char** names, double* total_ms, long long* launches, int cap);

/* Number of kernels this process has enqueued through the library. */
long long dgf_launch_count(void);

/*
 * Device-side errors.  Every wait of a kernel for one of its TMA copies is
 * bounded; when one runs out the kernel records bit 0 (a timeout) in the
 * library's status word on its device, waits (again bounded) for its copies
 * still in flight and stops, so that call's results are invalid.  The bit
 * is sticky: it is mirrored into a pinned host word (set up by the first
 * workspace call on the device, which must not come during a stream
 * capture), and every later entry point call on that device returns
 * DGF_ERR_TIMEOUT without launching anything until the bit is cleared.
 * dgf_forward_noalloc allocates nothing, so it sees the mirror only once
 * another entry point has set it up.
 *
 * dgf_device_status: reads the status word of the current device
 * (synchronous): 0 = no device-side error recorded; bit 0 = a bounded wait
 * ran out; -1 = the word could not be read.
 * dgf_clear_device_status: clears the word and its host mirror
 * (synchronous).
 * dgf_set_wait_polls: polls of a kernel's first wait on a copy (default and
 * maximum 2^22; the wait for copies still in flight after a timeout always
 * polls 2^22 times, so every copy lands before its buffer is reused).  A
 * test hook: 0 makes every first wait give up at once, which exercises the
 * timeout path without starving any copy.  Synchronous.  No counterpart in
 * the paper.
 */
int dgf_device_status(void);
dgf_status dgf_clear_device_status(void);
dgf_status dgf_set_wait_polls(long long polls);

/* Allows (1, default) or forbids (0) TMA staging of the low-resolution
 * tiles; with 0 every tile is staged with plain loads.  Results are
 * identical either way; this exists for testing the two paths. */
void dgf_set_tma(int on);

/* Allows (1, default) or forbids (0) the fused forward and backward: for r in {1, 2}, the
 * box mean of A, b, no guidance transform and an integer factor F with
 * F-pixel vectors of 8 or 16 bytes (F32: F = 2, 4; BF16/F16: F = 4, 8) and
 * I_h, O_h aligned to that vector, dgf_forward runs Eq. 1, both box means and
 * Eq. 2 (Sec. 3.2-3.3) in one kernel per high-resolution strip instead of a
 * low-resolution pass that writes Abar, bbar and a high-resolution pass that
 * reads them; likewise dgf_backward runs the backward's Eq. 1 pass and the
 * transposed upsampler (Algorithm 1's first two lines) in one kernel per
 * high-resolution strip for F32 F = 4 and BF16/F16 F = 8 with 16-byte
 * aligned dO_h, I_h, dI_h, writing the window statistics the low-resolution
 * backward reads.  The autotuner (when on) keeps whichever form is faster for
 * the call's key (its first call's sizes decide); untuned, the fused forms
 * serve r = 1 (at r = 2 on large images their redundant low-resolution
 * columns cost more than the saved Abar, bbar traffic).  The fused and
 * two-kernel forms give identical bits.  Either form needs the strip form
 * of the low-resolution pass (a pinned tile form keeps the two kernels). */
void dgf_set_fused(int on);

/* Allows (1, default) or forbids (0) the sliding-sum form of the
 * low-resolution kernels for 16-bit storage (BF16/F16, r in {1, 2, 4, 8},
 * the box mean of A, b): K1 (Eq. 1 and both box means, Sec. 3.2-3.3) and K4
 * (Algorithm 1 at low resolution) with running window sums over data shifted
 * by a per-strip constant, at a cost per pixel that does not grow with r.
 * Forbidden, 16-bit calls use the exactly centred forms FP32 storage always
 * uses.  The two agree within the 16-bit parity gates (the running sums
 * round differently); the sliding form's bits depend on its segment length
 * (autotune kinds 1 and 4) but not on the number of planes in a call. */
void dgf_set_lowres_slide(int on);

/* Allows (1, default) or forbids (0) the folded form of the grey guide
 * (dgf_options.guide_channels, Sec. 4.2 DGF_b): the high-resolution kernels
 * forming the channel mean of I_h in registers.  Forbidden, the grey guide
 * is formed in the workspace at both resolutions by streaming passes and the
 * layer runs on it.  Both forms form the mean the same way (FP32 sum over
 * the channels in order, one division); the backward's dI_h differs in
 * rounding (the folded form keeps the sum over output channels in FP32). */
void dgf_set_grey_fold(int on);

/* Allows (1, default) or forbids (0) the one-graph form of
 * dgf_backward_batched; forbidden, every batch runs the per-image chains.
 * Both give the same bits. */
void dgf_set_batched_graph_backward(int on);

/* Allows (1) or forbids (0, default) the plane-group pipeline of dgf_forward
 * and dgf_backward (no guidance transform, integer factor for the backward):
 * a call with 2 or more planes splits them into 2 or 3 groups and runs the
 * low-resolution kernels on a library stream of the greatest priority and
 * the high-resolution kernels on a second library stream, both forked from
 * and joined back to the caller's stream with events, so the low-resolution
 * pass of one group overlaps the high-resolution pass of another.  The call
 * stays asynchronous and stream-ordered on `stream` (and capturable in a
 * CUDA graph).  Results are identical either way.  Off by default: on
 * GB300 the low-resolution kernels are bound by the latency of their row
 * walks, so a group's pass takes nearly as long as the whole call's, and the
 * overlap does not pay for it.  No counterpart in the paper. */
void dgf_set_pipeline(int on);

/*
 * Options of the _opt entry points (NULL = the defaults of dgf_forward and
 * dgf_backward).
 *   mean_ab = 1 (default): the fast guided filter's box mean of A and b
 *             before upsampling (Abar, bbar), Algorithm 1 extended by f_mu^T;
 *   mean_ab = 0: A_l, b_l upsampled directly, the layer exactly as Sec. 3.2
 *             and Algorithm 1 print it.  Uses the warp-strip kernels for
 *             r in {1, 2} and the generic tiles otherwise; shapes are not
 *             autotuned in this mode.
 *   guide_channels = 0 (default) or C: the guide has the output's C
 *             channels (F the identity);
 *   guide_channels = n_I >= 1, n_I != C: the grey guide of Sec. 4.2 (DGF_b
 *             with differing channel counts): I_l (N x n_I x h_l x w_l) and
 *             I_h (N x n_I x h x w) are averaged over their channels in FP32,
 *             and that mean, held in FP32 (never rounded to dt), guides every
 *             one of the C output channels; dI_l, dI_h then have n_I channels
 *             (each the sum of the C channels' guide gradients / n_I).  Not
 *             with a guidance transform (g != NULL) and not in the batched or
 *             host-memory calls.  With an integer factor f in {2, 4, 8} and
 *             I_h, O_h (dO_h, dI_h) aligned to the vectors of the
 *             high-resolution tiles (16 bytes when w allows them, else 8;
 *             FP32 f = 8 is not among them), the high-resolution kernels
 *             read I_h's n_I channels and form the mean in registers: the
 *             forward writes O_h for all C channels of a tile from one pass
 *             over I_h, and the backward writes dI_h (from FP32 sums over
 *             the C channels) in the same pass that gathers the low-res
 *             gradients; only the low-res guide and its gradient go through
 *             the workspace.  Otherwise two streaming passes form the guide
 *             at both resolutions in the workspace before the layer and two
 *             more sum its gradient after it (with 16-bit dt the high-
 *             resolution stage then runs the general tile kernels).  The
 *             workspace (dgf_workspace_size_opt) covers the second form:
 *             the FP32 grey guide repeated over the C channels at both
 *             resolutions and its gradients.
 *   guide_low = 0 (default): with a guidance transform (g != NULL) the
 *             low-res guide is the f x f block mean of F(I_h) and I_l is not
 *             read;
 *   guide_low = 1: F applied to each guide on its own, G_l = F(I_l) and
 *             G_h = F(I_h) (Sec. 3.4 read literally).  Needs g and I_l
 *             (N x 3 x h_l x w_l); the backward may then return dI_l (through
 *             F at low resolution), and dW adds the low-res pixels' terms.
 *   coef = NULL (default): the backward recomputes the coefficients of the
 *             forward (Eq. 1 and the box mean) from its inputs;
 *   coef != NULL: device memory of dgf_coef_bytes(...) bytes, 256-byte
 *             aligned, owned by the caller: N x C x h_l x w_l FP32 pairs
 *             (Abar, bbar) (A_l, b_l with mean_ab = 0) and, with a guidance
 *             transform, from the next 256-byte boundaries the low-res guide
 *             G_l (N x 3 x h_l x w_l FP32) and the high-res guide F(I_h)
 *             (N x 3 x h x w FP32; not written with guide_low).
 *             dgf_forward_opt writes the call's values there (with the fused
 *             forward kernel then off: the two-kernel form, the same bits);
 *             dgf_backward_opt reads them as the forward's (the intermediate
 *             values Algorithm 1 takes from the forward pass) and skips the
 *             work that would only recompute them: its low-resolution K1
 *             pass where that pass produces nothing else, and with a
 *             guidance transform also the guide pass K5 and the evaluation
 *             of F per pixel in K3g (dgf_backward_reuses_coef tells when).  They
 *             must be what dgf_forward_opt wrote for the same inputs,
 *             weights, options and sizes; the backward's results are then
 *             the bits it gives without them.
 */
typedef struct {
    int mean_ab;
    int guide_channels;
    int guide_low;
    void* coef;
} dgf_options;

/* Bytes of the buffer dgf_options.coef points to for these sizes (g: with
 * a guidance transform, which adds the low-res and high-res guides); 0 for
 * invalid sizes.  Pure host function. */
size_t dgf_coef_bytes(int N, int C, int h_l, int w_l, int h, int w, const dgf_guide* g);

/* 1 when dgf_backward_opt with these sizes and options (coef aside) skips
 * work given the forward's coefficients (opt->coef): always with a guidance
 * transform or a folded grey guide; without them when the backward's
 * low-resolution pass would compute the coefficients alone (16-bit storage
 * with the sliding-sum kernels); 0 when that pass also produces the window
 * statistics the low-resolution backward reads (FP32 storage, r <= 2), where
 * the saved coefficients would only cost the forward a write.  A hint for
 * callers deciding whether to keep them: results are the same either way.
 * Pure host function (reads the autotuner's table). */
int dgf_backward_reuses_coef(int N, int C, int h_l, int w_l, int h, int w, int r, dgf_dtype dt,
                             const dgf_guide* g, const dgf_options* opt);

/* Workspace bytes of the _opt calls for these options (NULL = the defaults;
 * equals dgf_workspace_size then).  0 for invalid sizes or options. */
size_t dgf_workspace_size_opt(int N, int C, int h_l, int w_l, int h, int w, int r, dgf_dtype dt,
                              const dgf_guide* g, const dgf_options* opt);

dgf_status dgf_forward_opt(const void* p_l, const void* I_l, const void* I_h, void* O_h,
                           int N, int C, int h_l, int w_l, int h, int w, int r, float eps,
                           dgf_dtype dt, const dgf_guide* g, void* workspace, size_t ws_bytes,
                           dgf_stream_t stream, const dgf_options* opt);
dgf_status dgf_backward_opt(const void* dO_h, const void* p_l, const void* I_l, const void* I_h,
                            void* dp_l, void* dI_l, void* dI_h, float* dW,
                            int N, int C, int h_l, int w_l, int h, int w, int r, float eps,
                            dgf_dtype dt, const dgf_guide* g, void* workspace, size_t ws_bytes,
                            dgf_stream_t stream, const dgf_options* opt);

/*
 * One image of a batched backward call: the inputs of dgf_backward for one
 * image (C channels) and its gradient outputs, each output nullable (not
 * needed).  No guidance transform in the batched path.
 */
typedef struct {
    const void* dO_h;
    const void* p_l;
    const void* I_l;
    const void* I_h;
    void* dp_l;
    void* dI_l;
    void* dI_h;
    int C, h_l, w_l, h, w, r;
    float eps;
    const void* coef; /* NULL, or the image's coefficients from the forward (dgf_image.coef) */
} dgf_image_grad;

/*
 * Batched backward over images of different sizes, radii and factors
 * (Algorithm 1 per image, as dgf_backward with N = 1 and no guidance
 * transform).  With 16-bit storage, when every image's single call would run
 * the sliding low-res kernels and the strip K3 (the default for integer
 * factors 2, 4, 8 and radii 1, 2, 4, 8), the whole batch is one CUDA graph
 * of persistent kernels (dgf_set_batched_graph_backward): K1 nodes (one per
 * radius and lane width, images that want d I_h only) -> K3 nodes (one per
 * vector width and factor) -> K4 nodes (one per radius and lane width), each
 * node walking a flat list of every image's strip segments.  Otherwise each
 * image's chain of kernels runs on library-owned streams forked from and
 * joined back to `stream`.  Either way every image runs exactly its single
 * call's arithmetic, so the gradients equal the single calls' bit for bit
 * (the call is ordered on `stream` like any other).
 *   imgs:       n descriptors (host memory), 0 <= n <= DGF_MAX_BATCH;
 *               all tensors device memory in `dt`, NCHW with N = 1.
 *   workspace:  device memory of at least
 *               dgf_workspace_size_batched_backward(imgs, n, dt) bytes
 *               (0 for an invalid list), 256-byte aligned.
 * Errors as dgf_backward, with the failing image's index in the message.
 * Not under stream capture (the fork and join use library events).
 * No counterpart in the paper (batching machinery).
 */
size_t dgf_workspace_size_batched_backward(const dgf_image_grad* imgs, int n, dgf_dtype dt);
dgf_status dgf_backward_batched(const dgf_image_grad* imgs, int n, dgf_dtype dt, void* workspace,
                                size_t ws_bytes, dgf_stream_t stream);

/*
 * The batched calls with options (dgf_options; NULL = the defaults, the same
 * as dgf_forward_batched / dgf_backward_batched).  Only mean_ab is taken:
 * mean_ab = 0 runs every image as the layer Sec. 3.2 prints (A_l, b_l
 * upsampled without their box mean; Algorithm 1 without f_mu^T), each image's
 * kernel chain on one of the library streams forked from and joined back to
 * `stream` (no graph of persistent kernels); each image's outputs hold the
 * bits dgf_forward_opt / dgf_backward_opt give it with the same option.
 * guide_channels != 0 or guide_low != 0: DGF_ERR_UNSUPPORTED.  Workspace as
 * dgf_workspace_size_batched / dgf_workspace_size_batched_backward.
 */
dgf_status dgf_forward_batched_opt(const dgf_image* imgs, int n, dgf_dtype dt, void* workspace,
                                   size_t ws_bytes, dgf_stream_t stream, const dgf_options* opt);
dgf_status dgf_backward_batched_opt(const dgf_image_grad* imgs, int n, dgf_dtype dt, void* workspace,
                                    size_t ws_bytes, dgf_stream_t stream, const dgf_options* opt);

/*
 * Tile-shape autotuner.  When enabled (here, or DGF_AUTOTUNE=1 in the
 * environment), the first call for a new key (kernel, storage type, radius
 * or factor, vector width, guide type, and the size class of the low-res
 * plane: under 128 x 128 pixels or larger) times each candidate tile shape on that call's
 * own buffers and keeps the fastest; that call synchronises its stream and
 * must not be under stream capture (tuning is skipped while capturing).
 * Chosen shapes are used by every later call with the same key, tuned or
 * not, and are saved to the file DGF_TUNE_CACHE names (if any).  Each line
 * of that file is keyed by this library's cache version and the device name;
 * lines of another version or device are kept in the file but never used,
 * and malformed, truncated or out-of-range lines are skipped one by one (a
 * corrupt cache costs only a re-tune of the keys it held).  Results never
 * depend on the shape beyond FP32 rounding order.
 * dgf_autotune_entries: entries this device and library version would use.
 */
void dgf_autotune(int on);
int dgf_autotune_entries(void);
void dgf_autotune_reset(void);

/*
 * Pin one entry of the autotuner's table, as if tuning had chosen it: later
 * calls with that key use the shape (whether tuning is enabled or not), for
 * planes of both size classes.
 * Keys and shapes as the table stores them:
 *   kind 1 (K1 low-res coefficients) and 4 (K4 low-res backward): r = radius,
 *     F = vec = 0; guide_f32 = 1 for the guidance-transform path (FP32 guide);
 *     tiles: a = columns, b = rows of the coefficient region (a power of two
 *     in {64, 128, 256} and one of {16, 32, 64}); K1 with r <= 2 also takes
 *     warp strips: a = rows per segment in {8, 16, 24, 32, 48, 64, 128}, b = 0;
 *     with 16-bit storage both also take the sliding-sum strips
 *     (dgf_set_lowres_slide): a = output rows per segment in
 *     {8, 12, 16, 24, 32, 48, 64} (at least 2 r), b = -V with V the
 *     columns per lane (2, 4 or 8 for r <= 2; 4 for r in {4, 8}).
 *   kind 2 (K2 high-res apply): r = 0, F = integer factor (0: non-integer),
 *     vec = elements per vector; a = high-res rows per tile, b = 0.
 *   kind 3 (K3 high-res backward): as kind 2; a = low-res rows per segment
 *     of a warp strip (1 .. 256).
 *   kind 5 (fused forward, see dgf_set_fused): r = radius, F = factor,
 *     vec = guide_f32 = 0; a = low-res rows per segment (1 .. 256), or 0 to
 *     use the two-kernel forward for this key; b = 0.
 *   kind 6 (fused backward K1 + K3): r = radius, F = factor, vec = elements
 *     per vector, guide_f32 = 0; a as kind 5 (0: K1 and K3 as two kernels).
 * A shape the kernels are not built for is stored but ignored at plan time
 * (the default shape is used).  Returns DGF_ERR_INVALID for a key or shape
 * outside these ranges.  No counterpart in the paper: tuning machinery.
 */
dgf_status dgf_autotune_pin(int kind, dgf_dtype dt, int r, int F, int vec, int guide_f32, int a, int b);

/*
 * Forward pass that allocates nothing and takes no workspace.  The paper
 * has no counterpart; this exists for callers that cannot allocate device
 * memory when they call the layer (cudaMalloc may synchronise the device or
 * fail under memory pressure, so real-time loops and host frameworks that
 * own all device memory forbid it).  Same computation, arguments and
 * results as dgf_forward with F = identity (g = NULL), without the
 * workspace arguments.
 * Scratch: a fixed device array inside the library, dgf_noalloc_max_pairs()
 * low-resolution (Abar, bbar) pairs (8 MiB), held by every device that
 * loads the library until the process exits.  N*C*h_l*w_l above that
 * maximum returns DGF_ERR_UNSUPPORTED and enqueues nothing.
 * Set-up: the first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture on the device.
 * Sharing: every call uses the same array and leaves its last contents
 * there; each call overwrites all of it that it reads, so nothing needs
 * clearing, but calls whose kernels overlap on the device (different
 * streams, or different host threads) race on the array and must be
 * serialised by the caller.
 */
dgf_status dgf_forward_noalloc(const void* p_l, const void* I_l, const void* I_h, void* O_h,
                               int N, int C, int h_l, int w_l, int h, int w, int r, float eps,
                               dgf_dtype dt, dgf_stream_t stream);
size_t dgf_noalloc_max_pairs(void);

/*
 * Forward and backward of one batch whose tensors live in HOST memory
 * (Eq. 1-2 and Algorithm 1 as dgf_forward and dgf_backward compute them,
 * identity guide, box mean of A and b).  The call copies the inputs to the
 * device, runs the layer and copies the results back, pipelined over groups
 * of planes: while group g's kernels run, group g + 1's inputs travel
 * host -> device and group g - 1's results device -> host, on three
 * library-owned streams forked from and joined back to `stream`.  Planes
 * are independent, so every output plane holds the bits the device-memory
 * calls give for it.  No counterpart in the paper (I/O machinery).
 *   io:       host pointers (NCHW).  Inputs p_l, I_l (N x C x h_l x w_l) and
 *             I_h (N x C x h x w) are required; dO_h (N x C x h x w) is
 *             required when a gradient output is given.  Outputs, each
 *             nullable (not wanted): O_h (forward), dp_l, dI_l, dI_h
 *             (backward; with all three NULL the backward is not run).
 *             Pinned memory (cudaHostAlloc / cudaHostRegister) lets the
 *             copies overlap the kernels; pageable memory still works but
 *             the driver stages it and the overlap is lost.
 *   groups:   plane groups of the pipeline, 1 .. 16, or 0 for the default
 *             (min(N*C, 6)); clamped to N*C.
 *   device:   device memory of at least dgf_host_step_device_bytes(...)
 *             bytes, 256-byte aligned: the device copies of the eight
 *             tensors and the workspace of one group.  Owned by the caller;
 *             its contents after the call are unspecified.
 * The host buffers must stay valid, and the output buffers untouched, until
 * `stream` reaches the end of the call (cudaStreamSynchronize(stream)).
 * Errors as dgf_forward / dgf_backward; on an error in group g the groups
 * before it have been issued and `stream` is still joined to every library
 * stream.  Not under stream capture.
 */
typedef struct {
    const void* p_l;
    const void* I_l;
    const void* I_h;
    const void* dO_h;
    void* O_h;
    void* dp_l;
    void* dI_l;
    void* dI_h;
} dgf_host_step_io;

size_t dgf_host_step_device_bytes(int N, int C, int h_l, int w_l, int h, int w, int r, dgf_dtype dt,
                                  int groups);
dgf_status dgf_host_step(const dgf_host_step_io* io, int N, int C, int h_l, int w_l, int h, int w, int r,
                         float eps, dgf_dtype dt, int groups, void* device, size_t device_bytes,
                         dgf_stream_t stream);
/* dgf_host_step with options (NULL = the defaults): only mean_ab is taken
 * (mean_ab = 0: the layer as Sec. 3.2 prints it, every plane's outputs the
 * bits of dgf_forward_opt / dgf_backward_opt with that option);
 * guide_channels != 0 or guide_low != 0: DGF_ERR_UNSUPPORTED. */
dgf_status dgf_host_step_opt(const dgf_host_step_io* io, int N, int C, int h_l, int w_l, int h, int w, int r,
                             float eps, dgf_dtype dt, int groups, void* device, size_t device_bytes,
                             dgf_stream_t stream, const dgf_options* opt);

/* Releases cached graphs and tuning state (idempotent). */
void dgf_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* DGF_H */
