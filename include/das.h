/*
 * das.h -- C-ABI of the GB300 volumetric delay-and-sum (DAS) library.
 *
 * The library evaluates, on one GPU, the delay-and-sum image of the paper's
 * Sec. 2 ("Delay-and-sum"):
 *
 *   Eq. 1   tau_qmn = tau^tx_qn + ||p_n - r_m|| / c
 *   Eq. 2   x_bn    = sum_q sum_m w^tx_qn w^rx_mn y_bqm[tau_qmn] e^{+i 2 pi f_d tau_qmn}
 *
 * with y[tau] the linear interpolation between the samples k = floor(tau fs)
 * and k + 1 (Sec. 2, after Eq. 2), the batched channel tensor
 * y in C^{B x Q x M x K} with samples contiguous (Sec. 2, batched layout),
 * delays and receive weights computed in-kernel and never stored (Sec. 2,
 * problem scale; Sec. 3.1).  It also provides the adjoint map (image to
 * channel data) and the derivative with respect to the speed of sound c.
 *
 * Conventions (the paper leaves them open; the library fixes them so):
 *   - sample k is taken at t = k / fs (0-based);
 *   - diverging wave from virtual source v: tau^tx = (||p - v|| - ||v - o||) / c,
 *     t = 0 when the wave passes the reference point o (geometry.t0_ref);
 *     with options.t0_offset = 0: tau^tx = ||p - v|| / c;
 *   - plane wave with unit propagation direction d: tau^tx = d . (p - o) / c;
 *   - no transmit (photoacoustic, Sec. 2): tau^tx = 0;
 *   - IQ data: the focused sample is y[tau] e^{+i 2 pi f_d tau};
 *   - receive weight: with e = p - r_m, z = e . n_m, rho = |e x n_m|:
 *     1 if f_number <= 0, else 1 when z > 0 and rho^2 <= (1 + 1e-6) (z / 2F)^2,
 *     otherwise 0 (rectangular f-number aperture);
 *   - a term contributes only when 0 <= k <= K - 2.
 *
 * Memory: all "_dev" pointers are device pointers owned by the caller; "_host"
 * pointers are host memory owned by the caller.  The plan owns its own device
 * buffers (geometry, per-tile reference delays, channel-data relayout scratch)
 * and allocates them only in das_plan_create, das_plan_set_tuning (when a
 * tuning needs more scratch) and the first das_forward_host /
 * das_forward_host_many call; the other compute calls allocate nothing.  Calls are asynchronous on the given stream unless
 * stated otherwise; a plan must not be used by two streams at once.
 *
 * Errors: every function returns DAS_OK (0) or a DAS_ERR_* code.  Invalid
 * arguments are rejected before any launch.  das_last_error() returns a
 * thread-local text of the last failure.  Nothing aborts the process.
 */
#ifndef DAS_H
#define DAS_H

#ifdef __cplusplus
extern "C" {
#endif

#define DAS_OK 0
#define DAS_ERR_INVALID_ARG 1
#define DAS_ERR_CUDA 2
#define DAS_ERR_OOM 3
#define DAS_ERR_UNSUPPORTED 4
#define DAS_ERR_TIMEOUT 5

/* CUDA stream handle (same object as cudaStream_t; NULL is the legacy default stream). */
typedef struct CUstream_st *das_stream_t;

typedef struct das_plan das_plan_t;

/* Transmit kinds (Sec. 2, Eq. 1 footnote, and the photoacoustic remark). */
enum { DAS_TX_DIVERGING = 0, DAS_TX_PLANE = 1, DAS_TX_NONE = 2 };

/* Public channel-data / image element types. */
enum {
    DAS_SAMPLE_F32 = 0, /* real RF samples, float32; images float32 */
    DAS_SAMPLE_C64 = 1  /* complex IQ samples, interleaved float32 (re, im); images complex64 */
};

/* Storage of the channel data inside the plan after relayout (Sec. 3.3,
 * mixed-precision storage: 16-bit storage, float32 interpolation and sums). */
enum {
    DAS_STORE_F32 = 0,
    DAS_STORE_F16 = 1, /* half, with a float32 scale per (transmit, element) */
    DAS_STORE_BF16 = 2, /* bfloat16, with a float32 scale per (transmit, element) */
    DAS_STORE_E4M3 = 3, /* 8-bit float E4M3 (IQ data only; 8-bit storage is the paper's future work,
                           Sec. 6), the largest component of each (transmit, element) scaled to 448 */
    DAS_STORE_E5M2 = 4  /* 8-bit float E5M2 (IQ data only; two mantissa bits, a wider exponent range),
                           the largest component of each (transmit, element) scaled to 57344 */
};

/* Receive array (Sec. 2: receivers r_m, each with an origin and a direction). */
typedef struct {
    int n_elements;          /* M >= 1 */
    const double *positions; /* host, [M][3] metres */
    const double *normals;   /* host, [M][3] unit vectors, or NULL for +z */
    double t0_ref[3];        /* reference point o of the transmit time origin, metres */
} das_geometry_t;

/* Voxel grid: voxel (ix, iy, iz) at origin + spacing * (ix, iy, iz); images are
 * stored [b][iz][iy][ix] (x fastest), voxel index n = (iz * ny + iy) * nx + ix. */
typedef struct {
    int nx, ny, nz;
    double origin[3];
    double spacing[3];
} das_grid_t;

/* One transmit (observation q). */
typedef struct {
    int kind;          /* DAS_TX_* */
    double vec[3];     /* DIVERGING: virtual source (m); PLANE: unit propagation direction */
    const float *w_tx; /* host, [N] transmit weight per voxel (Sec. 2, precomputed w^tx), or NULL for 1 */
} das_tx_t;

typedef struct {
    int n_samples;   /* K >= 2 */
    int sample_type; /* DAS_SAMPLE_* of the public channel data and image */
    int storage;     /* DAS_STORE_* used inside the plan */
    int max_batch;   /* largest batch (frames per call) the plan reserves scratch for, >= 1 */
    int t0_offset;   /* 1: diverging-wave time origin at o (default reading); 0: paper footnote form */
} das_options_t;

/* Plan description returned by das_plan_info. */
typedef struct {
    long long n_voxels;       /* N */
    int n_elements;           /* M */
    int n_transmits;          /* Q */
    int n_samples;            /* K */
    int sample_type;
    int storage;
    int max_batch;
    long long device_bytes;   /* device memory held by the plan */
    double c;                 /* current speed of sound */
    long long kernel_launches; /* kernels this plan has launched so far */
    long long tc_mma_items;   /* tensor-core path: MMA sub-items issued so far, each an
                                 M 128 x N tc_mma_n x K 32 contraction (synchronises the device) */
    int tc_mma_n;             /* tensor-core path: MMA N of the last call (0: never used) */
} das_plan_info_t;

/* Kernel launch shape, set by the autotuner (das_plan_set_tuning). */
typedef struct {
    int frames_per_thread; /* frames accumulated per thread in the forward kernel (0: automatic) */
    int ctas_per_sm;       /* occupancy hint for persistent launches and the tensor-core
                              kernel (0: automatic); on the tensor-core path 2 also limits a
                              frame chunk to 112 frames so that two CTAs fit an SM, and 3 or 4
                              run CTAs of one builder group each with 48 frames per chunk
                              (automatic: 4 when a chunk holds 48 frames or fewer) */
    int staging;           /* 1: stage each (element, transmit) window of sample rows in shared
                              memory with bulk asynchronous copies; 0: read rows straight from
                              global memory (default) */
    int load_width;        /* how the kernels read sample rows from global memory: 0 (default)
                              column order, each row cut into 16-byte pieces stored along k so
                              that lanes with nearby delays share 128-byte lines (rows that are
                              not whole 16-byte pieces, and staged windows, use row order);
                              128 or 256: row order with loads of that many bits per lane */
    int tensor_cores;      /* 1: forward pass as a tensor-core contraction (Sec. 3.4 tile
                              reformulation on tcgen05 MMAs, IQ data with DAS_STORE_F16 or
                              DAS_STORE_BF16 only; the weights are rounded to the storage
                              type); 0: CUDA-core kernels (default).  Enabling it reserves
                              the operand scratch (2 x 2 bytes per sample and frame column). */
    int tc_chain;          /* tensor-core path: largest number of MMA sub-items summed in one
                              tensor-memory accumulation chain; at the first work-list end past it
                              the chain is added into the image in float32 and the next one starts
                              from zero, which keeps the tensor core's accumulation rounding
                              bias proportional to the chain rather than to all terms
                              (0: automatic, 1024 for plans of 4 or more transmits and one
                              chain per tile otherwise; -1: one chain per tile) */
    int voxels_per_thread; /* forward kernel for float32 IQ data in column order: 2 gives each
                              thread two voxels next to each other along x, which load three sample
                              rows for their four taps; 0 (default) or 1: one voxel per thread */
    int adjoint_rows;      /* das_adjoint: sample rows per CTA band (0: automatic); each CTA
                              accumulates one band of one element's rows in shared memory */
    int host_io;           /* das_forward_host / das_forward_host_many: 0 or 1 (default) copy the
                              batches through device staging buffers; 2: the kernels read the
                              channel data from, and write the image to, the caller's host memory
                              directly over the CPU-GPU link, no copy and no staging buffer: the
                              buffers must be page-locked (das_host_alloc, cudaHostAlloc,
                              cudaHostRegister) or, on systems where the GPU uses the host's page
                              tables, any host memory; others give DAS_ERR_INVALID_ARG */
} das_tuning_t;

/* Build a plan (Sec. 2 problem statement: grid, receivers, observations, c).
 * c: speed of sound (m/s, > 0); fs: sampling rate (Hz, > 0); f_demod:
 * demodulation frequency (Hz; 0 for RF); f_number: receive f-number (<= 0:
 * full aperture).  Copies the geometry to the device and reserves scratch for
 * options->max_batch frames.  Synchronous.  On failure *out is NULL. */
int das_plan_create(das_plan_t **out, const das_geometry_t *geometry, const das_grid_t *grid,
                    const das_tx_t *tx_list, int n_tx, double c, double fs, double f_demod,
                    double f_number, const das_options_t *options);

/* Release a plan and its device memory (synchronises the device).  NULL is accepted. */
void das_plan_destroy(das_plan_t *plan);

/* Change the speed of sound of the plan; the per-tile reference delays are
 * rebuilt on the stream of the next compute call.  No allocation. */
int das_plan_set_c(das_plan_t *plan, double c);

int das_plan_info(const das_plan_t *plan, das_plan_info_t *info);

int das_plan_set_tuning(das_plan_t *plan, const das_tuning_t *tuning);

/* Forward DAS (Eq. 2) for `batch` frames (1 <= batch <= max_batch).
 * y_dev: [batch][Q][M][K] samples of sample_type.  x_dev: [batch][N] image
 * (float32 for RF, complex64 for IQ), overwritten.  Runs the relayout of the
 * channel data into the plan's scratch (Sec. 3.2, batch-inner order, fused
 * with the 16-bit conversion of Sec. 3.3) and the DAS kernel. */
int das_forward(das_plan_t *plan, const void *y_dev, void *x_dev, int batch, das_stream_t stream);

/* das_forward with host buffers: copies y_host to the device, runs the
 * forward pass and copies the image back into x_host, then synchronises the
 * stream (with das_tuning_t.host_io = 2 the kernels read y_host and write
 * x_host directly instead, no copies: page-locked buffers only).  Uses device staging buffers, copy streams and events the plan
 * creates on first use (so the first call allocates).  Each copy is split
 * into up to 16 pieces on the plan's own copy streams, ordered with the work
 * on `stream`.  Pinned host memory is needed for full speed; memory from
 * das_host_alloc keeps it after long kernels. */
int das_forward_host(das_plan_t *plan, const void *y_host, void *x_host, int batch, das_stream_t stream);

/* das_forward_host over a sequence of n_batches batches of `batch` frames
 * each (no counterpart in the paper: host I/O around Eq. 2), with the copies
 * overlapped with the forward passes.  y_host[i] ([batch][Q][M][K] of
 * sample_type) and x_host[i] ([batch][N] image) are the host buffers of
 * batch i; the same input buffer may appear several times, an output buffer
 * may appear once only.  While the forward pass of batch i runs on `stream`,
 * the inputs of batch i + 1 are copied into a second device staging slot and
 * the image of batch i - 1 is copied out, each split into up to 16 pieces on
 * the plan's copy streams.  Returns when every image is in host memory.  The
 * first call allocates two staging slots (inputs and images for max_batch
 * frames each) and the copy events.  Every (y_host[i], x_host[i]) pair is
 * checked before any copy; NULL arrays or n_batches < 1 give
 * DAS_ERR_INVALID_ARG. */
int das_forward_host_many(das_plan_t *plan, const void *const *y_host, void *const *x_host, int n_batches,
                          int batch, das_stream_t stream);

/* Page-locked host memory for the host calls (no counterpart in the paper):
 * `bytes` rounded up to whole transparent huge pages, advised as huge pages,
 * touched and registered with CUDA (cudaHostRegister) for the current
 * device's context.  Host-to-device copies from small pinned pages lose much
 * of their speed right after long kernels (the GPU's translations of the host
 * pages are evicted); huge pages keep the copy at link speed.  Synchronous;
 * *ptr receives the address (64-byte aligned at least), or NULL on failure.
 * Free with das_host_free, which accepts only pointers from das_host_alloc
 * (DAS_ERR_INVALID_ARG otherwise) and NULL. */
int das_host_alloc(size_t bytes, void **ptr);
int das_host_free(void *ptr);

/* Adjoint DAS^H: the exact conjugate transpose of the linear map y -> x of
 * das_forward.  x_dev: [batch][N] (float32 / complex64); y_dev: [batch][Q][M][K]
 * of sample_type, overwritten (not accumulated).  For real RF data it is the
 * transpose; a complex64 x cannot be passed to an RF plan. */
int das_adjoint(das_plan_t *plan, const void *x_dev, void *y_dev, int batch, das_stream_t stream);

/* Derivative of the image with respect to c, contracted with a cotangent:
 * *dLdc_dev = Re sum_{b,n} conj(gx_bn) d x_bn / d c  (one double on the device).
 * Delays are recomputed, not stored.  With gx = 2 dL/d conj(x) (the gradient
 * PyTorch hands back for a real loss L of a complex image) this is dL/dc. */
int das_grad_c(das_plan_t *plan, const void *y_dev, const void *gx_dev, double *dLdc_dev, int batch,
               das_stream_t stream);

/* das_grad_c without any device allocation of its own.
 *
 * The paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory where they need the derivative (a fixed memory pool
 * that owns the device, a real-time loop that must not enter the allocator).
 * Same arguments and result as das_grad_c; the per-(voxel tile, frame chunk)
 * partial sums live in a 2 MiB array compiled into the library (262144
 * float64 slots, held by every GPU that loads the library until exit) instead
 * of in the plan.  Problems needing more slots (tiles x ceil(batch / frames per
 * thread)) are rejected with DAS_ERR_UNSUPPORTED before any launch.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * The address is kept for the life of the process: after a reset of the
 * device's primary context (cudaDeviceReset) the library must be unloaded
 * and loaded again before this entry point is called.
 * No slot needs clearing: each is written in the call before it is read.  All
 * calls share the one array, so calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  The plan's
 * channel-data scratch is used as in das_grad_c (allocated when the plan was
 * created): for IQ data, and for RF data of more than one frame.  Like every
 * call on a plan, calls on one plan must not overlap. */
int das_grad_c_static(das_plan_t *plan, const void *y_dev, const void *gx_dev, double *dLdc_dev, int batch,
                      das_stream_t stream);

/* Number of (q, m, n) terms of Eq. 2 that contribute (inside the aperture,
 * 0 <= k <= K - 2) for the plan's current c, counted on the device with the
 * kernels' own float32 decisions.  Synchronous; result in *count_host. */
int das_count_active(das_plan_t *plan, long long *count_host, das_stream_t stream);

/* Batches (the batched form): several plans -- grids of uneven size, element
 * and transmit counts, one sample type and storage -- and all their frames in
 * one persistent kernel launch.  The CTAs of the persistent grid take
 * (plan, frame chunk, voxel tile) items from an atomic work counter, heaviest
 * plans first, and run the forward tile body with that plan's arguments.  A
 * plan whose own tuning selects the tensor cores (das_plan_set_tuning,
 * tensor_cores = 1, f16 / bf16 IQ) is taken out of the work list and runs as
 * its own tensor-core launches (Sec. 3.4) in the same graph; that choice is
 * read when the batch is built (das_batch_create, das_batch_set_tuning).  The
 * per-plan relayouts, the counter reset and the launches are captured
 * once into a CUDA graph and replayed; a call with other data pointers
 * captures a new graph.  Up to 8 plans; frames[i] <= max_batch of plan i.
 * das_batch_create allocates the work list and may enlarge a plan's scratch;
 * das_batch_forward allocates nothing after its first call.  A batch keeps
 * pointers to its plans: destroy the batch first. */
typedef struct das_batch das_batch_t;
int das_batch_create(das_batch_t **out, das_plan_t *const *plans, const int *frames, int n_plans);
/* y_dev[i]: [frames[i]][Q_i][M_i][K_i]; x_dev[i]: [frames[i]][N_i], overwritten. */
int das_batch_forward(das_batch_t *batch, const void *const *y_dev, void *const *x_dev, das_stream_t stream);
/* frames_per_thread and ctas_per_sm (persistent CTAs per SM, 0: as many as fit) */
int das_batch_set_tuning(das_batch_t *batch, const das_tuning_t *tuning);
int das_batch_info(const das_batch_t *batch, int *frames_per_thread, int *n_items, int *kernels_per_launch);
void das_batch_destroy(das_batch_t *batch);

/* Waits for the stream and reports kernel-side failures recorded since the
 * last check: DAS_ERR_TIMEOUT when a kernel gave up a bounded wait (on a
 * staged copy, or inside the tensor-core pipeline) or the tensor-core path
 * met an item needing more sample windows than one work list holds (it
 * then left its outputs incomplete).  Clears the record. */
int das_plan_check(das_plan_t *plan, das_stream_t stream);

/* Test hook for the kernels' bounded waits (no counterpart in the paper:
 * failure handling around Eq. 2).  wait_ns (0 .. 1e10; 0 restores the default
 * of 1 s) limits every hand-off wait of the tensor-core pipeline, and the test
 * wait below in the staged kernel; the waits that let copies and MMAs still in
 * flight land before a CTA leaves keep their own 1 s limit.  probe = 1 makes
 * the first CTA of the next launches wait once on a shared-memory barrier that
 * nothing arrives on (the tensor-core kernel's MMA-issuing thread, or warp 1
 * of the staged kernel), so that the wait runs out after wait_ns: the CTA
 * records the failure in the plan's error word, drains, and leaves its part of
 * the output unwritten, and das_plan_check reports DAS_ERR_TIMEOUT.  Applies
 * to the calls issued after it; host only, synchronous, no allocation. */
int das_plan_set_wait_test(das_plan_t *plan, long long wait_ns, int probe);

/* Kernel timing for benchmarks.  With capacity > 0 the plan records a CUDA
 * event pair around the delay-and-sum kernel of each following das_forward
 * call, for up to `capacity` calls (capacity 0 switches it off).
 * das_plan_timing waits for the recorded events, returns the summed kernel
 * time in milliseconds and the number of timed launches, and starts over.
 * Events are created in das_plan_enable_timing, not in the timed calls. */
int das_plan_enable_timing(das_plan_t *plan, int capacity);
int das_plan_timing(das_plan_t *plan, double *ms_total, int *launches);

/* Text of the last error on the calling thread ("" if none). */
const char *das_last_error(void);

/* Library version string. */
const char *das_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DAS_H */
