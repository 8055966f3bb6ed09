/*
 * bdct.h -- C ABI of the GB300 (sm_103a) batched exact 2D DCT library.
 *
 * The operation (BRiDCT paper, Section 2.1):
 *   Eq. 1  (Q_n)_{kj} = alpha_k cos[(pi/n)(j + 1/2) k],
 *          alpha_0 = n^{-1/2}, alpha_k = (2/n)^{1/2} (k > 0).
 *   Eq. 2  forward  C(X) = Q_h X Q_w^T           (2D DCT-II)
 *          inverse  C^{-1}(Y) = Q_h^T Y Q_w       (2D DCT-III, the adjoint)
 *   Section 7.1: X may be rectangular, h x w.
 *   The round trip C^{-1}(C(X)) has exact result X (Section 2.1); it is
 *   computed with one read and one write of every element, the normalization
 *   folded between the forward core and its adjoint (Prop. 1, Eq. 4).
 *   The spectral direction is Prop. 1 with a general diagonal: the
 *   transform -- diagonal spectral operator -- inverse composition
 *   U^T Lambda U X = Q_h^T (Lambda o (Q_h X Q_w^T)) Q_w (Eq. 4), for instance
 *   the Poisson solve of a phase-unwrapping method (Section 1.1).
 *
 * Normalization (Section 2.1 names FFTW's REDFT10/REDFT01 pair):
 *   BDCT_NORM_ORTHO  Eq. 1-2 exactly.
 *   BDCT_NORM_NONE   forward  y_k = 2 sum_j x_j cos(pi (2j+1) k / (2n)) per axis,
 *                    inverse  x_j = y_0 + 2 sum_{k>=1} y_k cos(...) per axis,
 *                    so inverse(forward(X)) = 4hw X.  The round trip is the
 *                    normalized one and returns X under both settings.
 *
 * Data layout: every array is h rows by w columns of float32, row-major and
 * contiguous; a batch is `batch` such arrays back to back (stride h*w).
 * All data pointers are DEVICE pointers owned by the caller; the stream is a
 * cudaStream_t passed as void* (NULL = the legacy default stream).  Every
 * execution call is asynchronous on that stream and never allocates.
 *
 * Errors: every function returns a status (BDCT_OK = 0).  No exception, no
 * abort and no CPU fallback: if the device or the arguments do not fit, the
 * call fails with a status and does nothing.  bdct_status_string() names a
 * status; bdct_last_cuda_error() gives the CUDA error code behind the most
 * recent BDCT_ERR_CUDA on the calling thread.
 */
#ifndef BDCT_H
#define BDCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define BDCT_OK                    0
#define BDCT_ERR_INVALID_ARG       1  /* null pointer, dims < 1, bad enum value */
#define BDCT_ERR_UNSUPPORTED_SHAPE 2  /* shape outside what the requested path handles */
#define BDCT_ERR_KIND              3  /* direction not in the plan's kind mask */
#define BDCT_ERR_ALIGN             4  /* pointer not 16-byte aligned, or a stride not a multiple of 4 floats */
#define BDCT_ERR_ALIAS             5  /* input and output overlap partially */
#define BDCT_ERR_CUDA              6  /* a CUDA runtime call failed (see bdct_last_cuda_error) */
#define BDCT_ERR_ARCH              7  /* current device is not compute capability 10.3 */
#define BDCT_ERR_DEVICE_TIMEOUT    8  /* a bounded device-side wait expired */
#define BDCT_ERR_NO_MEMORY         9  /* plan-time device allocation failed */
#define BDCT_ERR_PATH             10  /* requested path cannot serve this shape */

/* -------------------------------------------------------- kinds (bitmask) */
#define BDCT_FORWARD   1u  /* 2D DCT-II, Eq. 2 left */
#define BDCT_INVERSE   2u  /* 2D DCT-III, Eq. 2 right */
#define BDCT_ROUNDTRIP 4u  /* C^{-1}(C(X)), normalized */
#define BDCT_SPECTRAL  8u  /* U^T Lambda U X, Prop. 1 / Eq. 4 (needs bdct_plan_set_spectral) */

/* ---------------------------------------------------------- normalization */
#define BDCT_NORM_ORTHO 0
#define BDCT_NORM_NONE  1

/* ------------------------------------------------------------------ paths
 * FP32       : CUDA-core FP32 fast factorization (even/odd DCT-II recursion,
 *              DCT-IV through a half-length complex FFT), passes fused on chip.
 * SPLIT_TC   : dense C X C^T on tcgen05 tensor cores, every operand split
 *              into three BF16 terms, six products accumulated in FP32.
 * SPLIT_HILO : the same with two BF16 terms and three products; its error is
 *              about 5e-6 relative, so it is reported but not accepted.
 * BF16       : single BF16 terms, one product; reported, never accepted.
 * AUTO       : the fastest path that meets the accuracy bar, per shape.     */
#define BDCT_PATH_AUTO       0
#define BDCT_PATH_FP32       1
#define BDCT_PATH_SPLIT_TC   2
#define BDCT_PATH_SPLIT_HILO 3
#define BDCT_PATH_BF16       4

typedef struct bdct_plan bdct_plan;

/* Create a plan for h = rows, w = cols on the CURRENT CUDA device.
 * kind: non-empty OR of BDCT_FORWARD / BDCT_INVERSE / BDCT_ROUNDTRIP /
 *       BDCT_SPECTRAL -- the directions the plan serves (tables are built
 *       only for those).
 * norm: BDCT_NORM_ORTHO or BDCT_NORM_NONE.   path: one of BDCT_PATH_*.
 * Supported shapes: FP32 path, any 1 <= rows, cols <= 8192 with cols a
 * multiple of 4; power-of-two sides 8..256 run fused on chip, other shapes
 * take separable passes through a plan-owned workspace.  Tensor-core paths:
 * rows and cols powers of two in 8..256.
 * The plan owns its device tables and workspace (Section 3.2: no allocation
 * or planning inside a transform).  Plan creation synchronizes the device.
 * On success *plan is set; on failure *plan is NULL and nothing leaks.      */
int bdct_plan_create(bdct_plan **plan, int rows, int cols, unsigned kind, int norm, int path);

/* Set the diagonal of the plan's spectral direction (Prop. 1, Eq. 4).
 * lambda: HOST array of rows x cols doubles, row-major, lambda[k*cols + l]
 * multiplying the orthonormal coefficient (k, l) (k along rows, l along
 * cols); copied, so the caller keeps ownership.  The plan must have been
 * created with BDCT_SPECTRAL in its kind (else BDCT_ERR_KIND).  The plan
 * keeps two FP32 tables computed from it in FP64 on the device: Lambda
 * itself, and Lambda folded with the squared scales (E Lambda E) for the
 * kernels that run the unscaled cores.  The spectral composition is the
 * normalized one under both normalizations (like the round trip).  May be
 * called again to replace the diagonal; it synchronizes the device, and no
 * work using the plan may be queued meanwhile.  A spectral execution before
 * the first call returns BDCT_ERR_INVALID_ARG.                              */
int bdct_plan_set_spectral(bdct_plan *plan, const double *lambda);

/* Numerical-range protection (Section 6 reports unnormalized intermediates
 * that overflow although the orthonormal result is representable, and
 * subnormal inputs that lose relative accuracy; Section 8 lists range
 * protection as future work).  With on != 0 every call of the plan scales
 * each array exactly by 2^-e, e the binary exponent of its largest
 * magnitude, transforms it, and scales the result back by 2^e (every
 * direction is linear, and a power-of-two scaling is exact while values stay
 * normal): the cores then never see magnitudes near FLT_MAX, and subnormal
 * inputs are transformed as normal numbers.  Costs two extra passes over the
 * output and one over the input; results equal the unprotected ones
 * wherever those stay within range.  Arrays whose largest magnitude is 0,
 * infinite or NaN are left unscaled.  The plan allocates 4 MiB of exponent
 * words (chunks of up to 2^20 arrays; a tiled call may hold at most 2^20
 * blocks, else BDCT_ERR_UNSUPPORTED_SHAPE).  on == 0 turns it off and frees
 * them.  No work using the plan may be queued.                             */
int bdct_plan_set_range_protection(bdct_plan *plan, int on);

/* Release a plan and its device memory.  The caller must ensure no work
 * using the plan is still queued.  NULL is accepted (no-op).               */
int bdct_plan_destroy(bdct_plan *plan);

/* Transform `batch` contiguous rows x cols float32 arrays from `in` to `out`
 * (device pointers, 16-byte aligned).  batch == 0 is a no-op.  in == out
 * (exact in-place) is allowed on every variant (the separable routes go
 * through the plan's workspace); any other overlap is BDCT_ERR_ALIAS.  The
 * input is left unchanged when in != out.                                  */
int bdct_forward(const bdct_plan *plan, const float *in, float *out, size_t batch, void *stream);
int bdct_inverse(const bdct_plan *plan, const float *in, float *out, size_t batch, void *stream);
int bdct_roundtrip(const bdct_plan *plan, const float *in, float *out, size_t batch, void *stream);

/* Same as above with the direction as an argument (one of the kind bits).
 * BDCT_SPECTRAL runs in one read and one write of every element on the fused
 * kernels of sides 8..32 and on the tensor-core route; the other shapes
 * compose it from the orthonormal forward, the diagonal and the inverse
 * (three passes over the output).                                          */
int bdct_execute(const bdct_plan *plan, unsigned kind, const float *in, float *out,
                 size_t batch, void *stream);

/* Tiled image view (Section 1.1: the motivating phase-unwrapping workload
 * transforms an image as many independent small blocks; Eq. 2 per block):
 * `in` is an img_rows x img_cols row-major image with
 * leading dimension ld_in floats; it is cut into (img_rows/rows) x
 * (img_cols/cols) independent rows x cols blocks, block (bi, bj) covering
 * rows bi*rows.. and columns bj*cols..; each block is transformed in place of
 * the same block of `out` (leading dimension ld_out).  img_rows and img_cols
 * must be multiples of the plan's rows and cols; ld_in and ld_out multiples
 * of 4.  in == out with ld_in == ld_out is exact in place; any other overlap
 * is BDCT_ERR_ALIAS.  The on-chip kernels support it: the fused FP32 and
 * tensor-core variants, and the dense route of small blocks (variant 2 with
 * both sides at most 64, e.g. 24 x 40 blocks); other plans return
 * BDCT_ERR_PATH.                                                            */
int bdct_execute_tiled(const bdct_plan *plan, unsigned kind, const float *in, float *out,
                       int img_rows, int img_cols, size_t ld_in, size_t ld_out, void *stream);

/* ------------------------------------------------------ host-buffer execution
 * End-to-end calls on HOST buffers (pinned memory gives overlap; pageable
 * memory works but each copy then blocks the host).  The paper times complete
 * calls including input copies (Sections 4.1-4.2) and names streaming
 * workloads with data transfers as future work (Section 8).
 * bdct_plan_set_host_staging allocates the plan's device staging (four slots
 * of two chunk_bytes buffers, rounded down to whole arrays, at least one) and
 * three private streams; call it once before the host entry points.
 * bdct_execute_host moves `batch` contiguous arrays from h_in through the
 * device and back to h_out in chunks: the host-to-device copy of one chunk,
 * the transforms of an earlier chunk and the device-to-host copy of one
 * before it overlap.  kinds[0..nkinds-1] (1..8 directions, each planned) are
 * applied in order to every chunk on the device, so an intermediate spectrum
 * never crosses the host link.  bdct_execute_tiled_host does the same for an
 * img_rows x img_cols host image (leading dimension img_cols) in bands of
 * whole block rows, through the tiled view.  Both are asynchronous on
 * `stream`: the host buffers must stay valid until the stream reaches the
 * end of the call; calls on one plan must not overlap.                      */
int bdct_plan_set_host_staging(bdct_plan *plan, size_t chunk_bytes);
int bdct_execute_host(const bdct_plan *plan, const unsigned *kinds, int nkinds, const float *h_in,
                      float *h_out, size_t batch, void *stream);
int bdct_execute_tiled_host(const bdct_plan *plan, const unsigned *kinds, int nkinds, const float *h_in,
                            float *h_out, int img_rows, int img_cols, void *stream);

typedef struct bdct_plan_info {
    int rows, cols;
    unsigned kind;
    int norm;
    int path;              /* resolved path (never AUTO) */
    int variant;           /* kernel family: 1 fused register tile, 2 separable passes (FFT line
                              engine, dense passes, or -- both sides at most 64 and no fused kernel
                              -- the dense operators applied in shared memory, one read and one
                              write), 3 tensor core on chip, 4 tensor-core separable passes */
    size_t workspace_bytes;
    size_t table_bytes;
} bdct_plan_info;

int bdct_plan_get_info(const bdct_plan *plan, bdct_plan_info *info);

/* The separable routes (variants 2 and 4: two passes over every array, the
 * first one writing the transposed intermediate to the plan's workspace; the
 * paper's two-pass structure of Eq. 2) process the batch in chunks of whole
 * arrays.  Set the chunk to about `bytes` (at least one array): the workspace
 * is reallocated to match.  A chunk that fits in L2 lets the second pass read
 * the intermediate from L2 instead of HBM, while every chunk costs two pass
 * launches with their ramp-up and drain (which measured the larger effect).
 * The default is 256 MiB; the ragged autotuner picks it per shape class.
 * No work using the plan may be queued.  Other variants (and the on-chip
 * dense route of small arrays) keep no workspace and ignore the call
 * (BDCT_OK).                                                               */
int bdct_plan_set_chunk_bytes(bdct_plan *plan, size_t bytes);

/* Synchronize the device and return the plan's device-side status: BDCT_OK,
 * or BDCT_ERR_DEVICE_TIMEOUT if a bounded wait inside one of the plan's
 * kernels gave up since the last clear (the kernel then stopped early and its
 * output is incomplete).  clear != 0 resets the word.  Host errors are
 * returned as usual.                                                         */
int bdct_plan_device_status(const bdct_plan *plan, int clear);

/* ------------------------------------------------------------ ragged batches
 * A batch of arrays of mixed shapes (the paper transforms one array per call
 * and loops over batches in C, Section 3.2).  Array i has rows[i] x cols[i]
 * elements, contiguous and row-major, starting in_off[i] and out_off[i]
 * floats after the base pointers given at execution (offsets multiples of 4;
 * arrays must not overlap, except an array whose in and out spans coincide).
 * Arrays are grouped by shape; each group gets a plan whose path, when `path`
 * is BDCT_PATH_AUTO, is the fastest of the accepted candidates (FP32, and the
 * on-chip split-BF16 tensor-core path where it exists; for shapes on the
 * separable route, its workspace chunk of 64, 128 or 256 MiB) timed on scratch
 * arrays at creation -- or read from the file named by the environment
 * variable BDCT_TUNE_CACHE, to which new choices are appended.  Creation
 * allocates, synchronizes and runs those timing launches.
 * Execution launches one persistent kernel (or, on the separable routes, one
 * pair of pass kernels per chunk) per shape class, reading the arrays through
 * device offset tables, from a CUDA graph captured on the first call for each
 * (kind, in_base, out_base) and replayed afterwards on `stream`, the largest
 * class first.
 * The first call for new pointers should not itself run inside a stream
 * capture.  Calls on the same ragged plan must not overlap on the GPU.      */
typedef struct bdct_ragged bdct_ragged;

typedef struct bdct_ragged_class {
    int rows, cols;
    size_t count;              /* arrays of this shape */
    int path;                  /* chosen path */
    int variant;               /* kernel family, as in bdct_plan_info */
    double tuned_us_per_array; /* measured at creation (0 if not timed) */
    size_t chunk_bytes;        /* separable routes: workspace chunk chosen (0: none) */
} bdct_ragged_class;

int bdct_ragged_create(bdct_ragged **ragged, size_t n, const int *rows, const int *cols,
                       const size_t *in_off, const size_t *out_off, unsigned kind, int norm, int path);
int bdct_ragged_execute(bdct_ragged *ragged, unsigned kind, const float *in_base, float *out_base,
                        void *stream);
int bdct_ragged_destroy(bdct_ragged *ragged);
/* Number of shape classes (or a negated status). */
int bdct_ragged_num_classes(const bdct_ragged *ragged);
/* Classes are ordered by total elements, largest first. */
int bdct_ragged_class_info(const bdct_ragged *ragged, int index, bdct_ragged_class *info);

/* Allocation-free transform, for callers that cannot allocate device memory
 * (their memory is owned by another allocator, or they must avoid the device
 * synchronization that allocation and release can cause, or their footprint
 * must be fixed when the library loads).  No plan is needed and nothing is
 * allocated: the separable dense route (FP64-generated operator matrices,
 * then a row pass and a column pass through an intermediate buffer) keeps
 * all of its scratch in one file-scope device array of 8 MiB, which every
 * GPU that loads the library holds until the process exits.
 * Arguments as in bdct_plan_create + bdct_execute: kind is ONE of
 * BDCT_FORWARD / BDCT_INVERSE / BDCT_ROUNDTRIP; in and out are 16-byte
 * aligned device pointers to `batch` contiguous rows x cols arrays (equal or
 * disjoint).  Limits: 1 <= rows, cols <= 512, cols a multiple of 4; larger
 * sides return BDCT_ERR_UNSUPPORTED_SHAPE.  Batches larger than the scratch
 * holds are processed in chunks.
 * The first call on each device looks up the array's device address once
 * (cudaGetSymbolAddress with that device current); make that first call
 * before any stream capture.  Every call shares the one array and leaves its
 * contents behind; each call rewrites everything it reads, so nothing needs
 * to start at zero, but calls that overlap on the GPU (different streams,
 * or host threads racing) corrupt each other's scratch and must be
 * serialized by the caller.
 * The paper has no counterpart to this entry point.                          */
int bdct_execute_noalloc(int rows, int cols, unsigned kind, int norm, const float *in, float *out,
                         size_t batch, void *stream);

/* Self-test of the bounded device-side wait: launches one thread that waits
 * on a barrier nothing completes, with a limit of limit_us microseconds
 * (1..2000000), and returns the status it recorded -- BDCT_ERR_DEVICE_TIMEOUT
 * when the bounded wait behaves, with the CUDA context still usable.  No
 * counterpart in the paper: it tests the library's failure detection.       */
int bdct_selftest_wait_timeout(unsigned int limit_us);

/* Name of a status code (static string, never NULL). */
const char *bdct_status_string(int status);

/* CUDA error code behind the calling thread's most recent BDCT_ERR_CUDA. */
int bdct_last_cuda_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int bdct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BDCT_H */
