/*
 * triot.h -- C ABI of the GB300 (sm_103a) TRIOT hot path.
 *
 * Joint iteration over dense row-major tensors of different shapes whose rank is known
 * only at run time, with the index tuple visible to the operation: Heyl & Serang,
 * "TRIOT: Faster tensor manipulation in C++11" (arXiv 1608.00099).  Three operations:
 *   embed / crop  -- copy into a larger zero-padded tensor and back (Section 3,
 *                    benchmark 1; Algorithm 13),
 *   product       -- y[t] *= x[t] over the tuples shared by both shapes (Section 3,
 *                    benchmark 2; apply_tensors of Algorithm 9),
 *   moment        -- the tuple-weighted sum  m_i = sum_t p[t] * t_i  (Algorithms 10, 11).
 *
 * Conventions shared by every call
 *   - Tensors are dense, contiguous and row-major.  Data pointers are DEVICE pointers
 *     owned by the caller; 16-byte alignment is recommended (it enables 128-bit
 *     accesses) but not required beyond the element size.
 *   - Shapes are HOST arrays of `rank` int64 extents, read during the call only.
 *     1 <= rank <= TRIOT_MAX_RANK.  Extents may be 0 (empty iteration) or 1.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *     enqueue work and return without synchronising; they allocate no memory, so they
 *     may be captured in a CUDA graph.
 *   - Every call returns a triot_status.  On failure nothing has been enqueued and
 *     triot_last_error() describes the problem (thread-local string).
 *   - dtype codes: TRIOT_F64, TRIOT_F32, TRIOT_BF16, TRIOT_F16.  IEEE round-to-nearest-
 *     even throughout; denormals are kept (no flush to zero).
 */
#ifndef TRIOT_H
#define TRIOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRIOT_MAX_RANK 24

typedef enum triot_dtype {
  TRIOT_F64 = 0,
  TRIOT_F32 = 1,
  TRIOT_BF16 = 2,
  TRIOT_F16 = 3
} triot_dtype;

typedef enum triot_status {
  TRIOT_OK = 0,
  TRIOT_ERR_RANK = 1,      /* rank < 1 or rank > TRIOT_MAX_RANK                        */
  TRIOT_ERR_SHAPE = 2,     /* negative extent, or a source not inside its target         */
  TRIOT_ERR_NULL = 3,      /* a required pointer is NULL (data may be NULL when empty)   */
  TRIOT_ERR_DTYPE = 4,     /* unknown dtype code                                         */
  TRIOT_ERR_WORKSPACE = 5, /* workspace too small or misaligned                          */
  TRIOT_ERR_ALIAS = 6,     /* x and y are the same pointer (they must not overlap)       */
  TRIOT_ERR_CUDA = 7,      /* a CUDA runtime call or kernel launch failed                */
  TRIOT_ERR_ARG = 8,       /* any other invalid argument (flags, sizes, tuning values)   */
  TRIOT_ERR_DEVICE = 9     /* a device-side guard tripped (see triot_device_status)      */
} triot_status;

/* embed flag: y is already all zero; write only x's tuples (skip the pad). */
#define TRIOT_EMBED_NOPAD 1u

/* Thread-local description of the last failure of a call made by this thread. */
const char* triot_last_error(void);
/* Library version string, e.g. "triot-gb300 1.0 sm_103a". */
const char* triot_version(void);

/*
 * triot_embed -- zero-padded copy at the origin.
 *   Section 3 benchmark 1 run in reverse (the abstract's "copying data from one tensor to
 *   another larger, zero padded tensor"): for every tuple t of y's shape,
 *       y[t] = x[t]  if t_i < xshape[i] for all i,   y[t] = +0.0 (all bits zero) otherwise.
 *   Requires xshape[i] <= yshape[i] for every i (else TRIOT_ERR_SHAPE), the bounds check
 *   check_tensor_pack_bounds performs once per call (Algorithm 8).
 *   x: device, rank-`rank` tensor of xshape, read only.  y: device tensor of yshape,
 *   written in full (with TRIOT_EMBED_NOPAD only x's tuples are written).
 *   The operation moves bits: it is bit-exact for every dtype (the dtype only fixes the
 *   element size).  x and y must not overlap.
 */
int triot_embed(int rank, const int64_t* xshape, const void* x, const int64_t* yshape,
                void* y, int dtype, unsigned flags, void* stream);

/*
 * triot_crop -- the inverse of embed (Algorithm 13, benchmark 1):
 *       x[t] = y[t]  for every tuple t of x's shape.
 *   Requires xshape[i] <= yshape[i].  x (device, written in full) and y (device, read)
 *   must not overlap.  Bit-exact for every dtype.
 */
int triot_crop(int rank, const int64_t* xshape, void* x, const int64_t* yshape,
               const void* y, int dtype, void* stream);

/*
 * triot_product -- in-place element-wise product over the shape intersection:
 *       y[t] = y[t] * x[t]  for every tuple t with t_i < min(xshape[i], yshape[i]);
 *   y elsewhere is untouched (Section 3 benchmark 2 visits "only tuple indices shared by
 *   both"; the write goes to the destination only, as apply_tensors in Algorithm 9).
 *   f64/f32: one IEEE multiply.  bf16/f16: the exact product of the stored values,
 *   rounded once to the storage type.  x (device, read) and y (device, read-write) must
 *   not overlap (the __restrict contract of Section 4).
 */
int triot_product(int rank, const int64_t* xshape, const void* x, const int64_t* yshape,
                  void* y, int dtype, void* stream);

/*
 * triot_convolve -- naive multidimensional convolution (Algorithms 14 and 15; Section 3,
 *   benchmark 4): out[t] = sum of a[u] * b[t - u] over the tuples u of a's shape for which
 *   t - u is a tuple of b's shape, for every tuple t of the result shape
 *   ashape + bshape - 1 (dense row-major, written entirely; an axis of extent 0 in a or b
 *   gives an all-zero result on that extent).  dtype must be TRIOT_F64.  Each product is
 *   rounded, then the products of an output are summed in a fixed order (32 partial sums
 *   over the outermost axis, combined pairwise), so the result differs from the paper's
 *   scatter order only by rounding and is identical from run to run.  out must not overlap
 *   a or b.
 */
int triot_convolve(int rank, const int64_t* ashape, const void* a, const int64_t* bshape,
                   const void* b, void* out, int dtype, void* stream);

/*
 * triot_apply -- an elementwise operation over three tensors of different shapes, visiting
 *   every tuple t of x's shape (Algorithm 9's apply with several tensors).  The fixed set of
 *   operations:
 *     TRIOT_APPLY_XPYXMZ   x[t] <- x[t] + y[t] * x[t] - z[t]   (Section 3, benchmark 3)
 *   y and z must contain x's shape on every axis (TRIOT_ERR_SHAPE otherwise); each tensor is
 *   addressed with its own shape.  Evaluated left to right, each operation rounded to nearest
 *   even (no fused multiply-add): in double for TRIOT_F64, in float for TRIOT_F32, and in
 *   float for TRIOT_BF16 / TRIOT_F16 with one final rounding to the storage format.
 *   x is read and written in place; y and z are read; none may overlap another.
 */
#define TRIOT_APPLY_XPYXMZ 1
int triot_apply(int op, int rank, const int64_t* xshape, void* x, const int64_t* yshape,
                const void* y, const int64_t* zshape, const void* z, int dtype, void* stream);

/*
 * Views (Section 4: a slice references its tensor and adds a bias -- the flat index of its
 * start tuple computed with the tensor's own shape -- to every flat index).  `ystart` is a
 * HOST array of rank non-negative starts; the window of y is the tuples ystart + t.
 *
 * triot_embed_at  -- y[ystart + t] = x[t] for every tuple t of x's shape; every other element
 *   of y is set to +0 unless flags has TRIOT_EMBED_NOPAD (then it is left untouched).
 *   Requires ystart + xshape <= yshape on every axis (TRIOT_ERR_SHAPE otherwise).  Without
 *   NOPAD two kernels are enqueued (the pad over all of y, then the copy).
 * triot_crop_at   -- x[t] = y[ystart + t] for every tuple t of x's shape (the inverse: the
 *   extraction step after a zero-padded transform).  Same requirement.
 * triot_product_at -- y[ystart + t] *= x[t] for every tuple t of x's shape with
 *   ystart + t inside y (the intersection of x's shape with y's remainder yshape - ystart);
 *   requires ystart <= yshape.  Rounding as triot_product.
 * Other arguments, errors and aliasing rules as the whole-tensor calls (x and y must not
 * overlap anywhere in their containers).
 */
int triot_embed_at(int rank, const int64_t* xshape, const void* x, const int64_t* yshape, void* y,
                   const int64_t* ystart, int dtype, unsigned flags, void* stream);
int triot_crop_at(int rank, const int64_t* xshape, void* x, const int64_t* yshape, const void* y,
                  const int64_t* ystart, int dtype, void* stream);
int triot_product_at(int rank, const int64_t* xshape, const void* x, const int64_t* yshape, void* y,
                     const int64_t* ystart, int dtype, void* stream);

/*
 * Windows on both sides (Section 4: views over the intersecting support of two tensors, so
 * that e.g. the product of two PMFs with different supports runs without copies).  `ext` is
 * the window's extents; `xstart` / `ystart` (HOST arrays of rank non-negative starts) place
 * it in the containers x (xshape) and y (yshape), each addressed with its own shape.
 * triot_copy_views    -- y[ystart + t] = x[xstart + t] for every tuple t of ext (bit-exact).
 * triot_product_views -- y[ystart + t] = y[ystart + t] * x[xstart + t] (rounded as
 *   triot_product).
 *   Both windows must lie inside their containers (TRIOT_ERR_SHAPE otherwise); x and y must
 *   not overlap; the rest of y is untouched.
 * triot_product_support -- the product of two tensors placed on a common integer grid:
 *   x covers the tuples xorigin + [0, xshape), y covers yorigin + [0, yshape) (origins are
 *   HOST arrays of rank signed values, |origin| < 2^62); y is multiplied by x over the
 *   tuples both cover (none: nothing happens), i.e. triot_product_views on the window
 *   [max(xorigin, yorigin), min(xorigin + xshape, yorigin + yshape)).
 */
int triot_copy_views(int rank, const int64_t* ext, const int64_t* xshape, const void* x,
                     const int64_t* xstart, const int64_t* yshape, void* y, const int64_t* ystart,
                     int dtype, void* stream);
int triot_product_views(int rank, const int64_t* ext, const int64_t* xshape, const void* x,
                        const int64_t* xstart, const int64_t* yshape, void* y, const int64_t* ystart,
                        int dtype, void* stream);
int triot_product_support(int rank, const int64_t* xshape, const void* x, const int64_t* xorigin,
                          const int64_t* yshape, void* y, const int64_t* yorigin, int dtype, void* stream);

/*
 * triot_moment_workspace_size -- bytes of device workspace triot_moment needs for this
 *   shape and dtype (per-block partial sums).  Writes *bytes; never fails for valid
 *   arguments.  The size depends only on (rank, shape, dtype) and the tuning in force.
 */
int triot_moment_workspace_size(int rank, const int64_t* shape, int dtype, size_t* bytes);

/*
 * triot_moment -- tuple-weighted first moments (Algorithm 11 with one weight tensor,
 *   the tuple made visible as in Algorithm 10; tuples are zero-based):
 *       out[i]    = sum over tuples t of shape  p[t] * t_i     (i = 0 .. rank-1)
 *       out[rank] = sum over tuples t of shape  p[t]            (the mass)
 *   p: device tensor, read only.  out: DEVICE array of rank+1 doubles, written.
 *   workspace: device scratch of at least triot_moment_workspace_size() bytes, 16-byte
 *   aligned, owned by the caller; its contents on entry are ignored.
 *   Accumulation: f64 input in two's-complement fixed point, exact within windows of at
 *   most 1024 elements per thread and rounded to f64 once per window (error at most
 *   2^-52 times the window's largest |p| per element).  f32/bf16/f16 input in f32: with
 *   compensated sums per thread when the innermost extent exceeds 16, otherwise (trailing
 *   axes forming blocks) with plain f32 sums of at most 64 terms per thread and window,
 *   added across each warp into compensated f32 totals (error below about 5.6e-6 of
 *   sum |p[t]| t_i); finite f32 data whose partial sums exceed the f32 range give inf.
 *   Block partials are combined by a second kernel in fixed point, independent of their
 *   order, so results are bit-identical from run to run.  Two kernels are enqueued on
 *   `stream`.
 */
int triot_moment(int rank, const int64_t* shape, const void* p, int dtype, double* out,
                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * triot_moment_noalloc -- the same result as triot_moment, for callers that cannot
 *   allocate device memory and so cannot provide a workspace (for example code that runs
 *   where cudaMalloc is forbidden or would synchronise the device, or an application
 *   whose device memory is owned entirely by its own pool).  The paper has no
 *   counterpart: this is a deployment convenience of this library.
 *   The per-block partial sums go to a fixed scratch array of
 *   TRIOT_MOMENT_NOALLOC_MAX_DOUBLES doubles (512 KiB) that lives in the library image;
 *   every GPU that loads the library holds it until the process exits.  The call itself
 *   allocates nothing (no cudaMalloc, no library allocator).
 *   Arguments as triot_moment without the workspace.  Fails with TRIOT_ERR_WORKSPACE,
 *   and enqueues nothing, when the launch would need more partials than the scratch
 *   holds: the partials number grid * (effective rank + 1), where the grid is at most
 *   SMs x resident CTAs per SM of the chosen moment kernel (or x the tuned ctas_per_sm);
 *   the default plans of every workload this library measures fit (for example 9^8 in f64
 *   and 2^24 elements of rank 24 in f32), a forced ctas_per_sm of 32 at rank 24 does not.
 *   The first call on a device looks up the scratch's device address (once, with that
 *   device current) and keeps it for the life of the process: make that first call before
 *   any stream capture, and do not use this call across a cudaDeviceReset (the address it
 *   keeps belongs to the context the reset destroys).  All calls share the
 *   one scratch array, which keeps the last call's contents: calls whose kernels may
 *   overlap on the GPU (different streams without ordering) race on it.
 */
#define TRIOT_MOMENT_NOALLOC_MAX_DOUBLES 65536
int triot_moment_noalloc(int rank, const int64_t* shape, const void* p, int dtype, double* out,
                         void* stream);

/*
 * triot_moment_product_workspace_size -- bytes of device workspace triot_moment_product
 *   needs for these shapes and dtype.  Writes *bytes.
 */
int triot_moment_product_workspace_size(int rank, int ntensors, const int64_t* const* shapes,
                                        int dtype, size_t* bytes);

/*
 * triot_moment_product -- the tuple-weighted moment of a product of tensors over the
 *   tuples their shapes share (Algorithm 11 weights the tuple by x[t]*y[t]*z[t]; with two
 *   tensors out[rank] is the inner product over the shared tuples of Section 3's second
 *   benchmark), without forming the product in memory:
 *       I         = elementwise minimum of the shapes
 *       w[t]      = x_0[t] * x_1[t] * ... * x_{n-1}[t], left to right
 *       out[i]    = sum over tuples t of I  w[t] * t_i     (i = 0 .. rank-1, zero-based)
 *       out[rank] = sum over tuples t of I  w[t]
 *   ntensors: 1 .. 4.  shapes[k]: HOST array of rank extents of tensor k; tensors[k]:
 *   its DEVICE data (dense row-major, read only), all of the same dtype.  The products are
 *   rounded to nearest even in double for TRIOT_F64 and in float for TRIOT_F32, TRIOT_BF16
 *   and TRIOT_F16 (whose values float holds exactly).  out: DEVICE array of rank+1 doubles.
 *   workspace: device scratch of at least triot_moment_product_workspace_size() bytes,
 *   16-byte aligned.  Sums are fixed point, exact within windows of at most 1024 elements
 *   per thread (error at most 2^-52 times the window's largest |w| per element for f64
 *   tensors, 2^-48 for the others); when the last axis of I is shorter than 8 (a CTA-tiled
 *   kernel), relative to the largest |w| the CTA has met so far (at most 2^-52 of it per
 *   element, every dtype).  Partials are combined independently of their order, and a
 *   non-finite weight propagates as in a plain sum.  Two kernels are enqueued.
 *   Errors: TRIOT_ERR_ARG (ntensors outside 1..4), TRIOT_ERR_RANK, TRIOT_ERR_SHAPE
 *   (negative extent, extent >= 2^31), TRIOT_ERR_NULL, TRIOT_ERR_DTYPE,
 *   TRIOT_ERR_WORKSPACE, TRIOT_ERR_CUDA.  An empty intersection writes zeros.
 */
int triot_moment_product(int rank, int ntensors, const int64_t* const* shapes,
                         const void* const* tensors, int dtype, double* out, void* workspace,
                         size_t workspace_bytes, void* stream);

/*
 * triot_nonzero_bbox -- the bounding box of the nonzero entries of a product of tensors
 *   (Section 2: with the tuple visible to the operation, "the nonzero bounding box for the
 *   element-wise product of two tensors" is a reduction over the tuples):
 *       I        = elementwise minimum of the shapes
 *       counted  = the tuples t of I with x_k[t] != 0 for every k (the support of the
 *                  product as real functions: IEEE comparison with zero, so NaN and
 *                  infinities count, +0 and -0 do not; nothing is rounded)
 *       out[2i]  = least t_i over the counted tuples, out[2i+1] = greatest t_i (i = 0 ..
 *                  rank-1, zero-based), out[2 rank] = the number of counted tuples
 *   With nothing counted (or an empty I) every out[2i] = 0 and out[2i+1] = -1, count 0.
 *   ntensors: 1 .. 4.  shapes[k]: HOST array of rank extents; tensors[k]: DEVICE data of one
 *   dtype (dense row-major, read only).  out: DEVICE array of 2 rank + 1 int64.  workspace:
 *   device scratch of at least triot_nonzero_bbox_workspace_size() bytes, 16-byte aligned
 *   (its contents on entry are ignored).  Exact: min / max / count do not depend on the
 *   order of the tuples, so results are identical from run to run.  Two kernels are
 *   enqueued.  Errors as triot_moment_product.
 */
int triot_nonzero_bbox_workspace_size(int rank, int ntensors, const int64_t* const* shapes, int dtype,
                                      size_t* bytes);
int triot_nonzero_bbox(int rank, int ntensors, const int64_t* const* shapes, const void* const* tensors,
                       int dtype, int64_t* out, void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------ batched launch */

/*
 * One pair of the batched pipeline: x (xshape) is embedded at the origin of a zero-padded
 * y (yshape), then y[t] *= x[t] over x's shape, then the moment of y is written to
 * moment_out[0 .. rank] (rank moments then the mass, as triot_moment).  All pointers are
 * device pointers owned by the caller.  Section 4: independent problems are partitioned
 * across processors with no shared state.
 */
typedef struct triot_batch_desc {
  int rank;                           /* 1 .. TRIOT_MAX_RANK                         */
  int64_t xshape[TRIOT_MAX_RANK];
  int64_t yshape[TRIOT_MAX_RANK];
  const void* x;                      /* device, read                                 */
  void* y;                            /* device, written in full                      */
  double* moment_out;                 /* device, rank + 1 doubles                     */
} triot_batch_desc;

/* Launch geometry of a kernel family; zero fields mean "use the tuned or default value". */
typedef struct triot_tune {
  int threads;      /* threads per CTA (multiple of 32, 64 .. 1024)                       */
  int tile_elems;   /* elements of the iteration space one CTA handles per tile          */
  int ctas_per_sm;  /* resident CTAs per SM for persistent launches (1 .. 8)              */
  int unroll;       /* vectors in flight per thread (1 .. 8)                              */
} triot_tune;

typedef struct triot_plan triot_plan;

/* batch plan modes */
#define TRIOT_BATCH_FUSED 0       /* one persistent kernel: embed+product+moment per tile */
#define TRIOT_BATCH_PHASED 1      /* persistent embed, product, moment phases            */

/*
 * triot_batch_plan_create -- validate `n` descriptors (all of one dtype: TRIOT_F32,
 *   TRIOT_F64, TRIOT_BF16 or TRIOT_F16), build the device work list (descriptors, tile
 *   prefix sums, moment slots) and return an opaque plan.  This call allocates device
 *   memory (once); running the plan does not.  Geometry: tile_elems (elements of a work
 *   tile, 1 .. 2^20) and ctas_per_sm (1 .. 32) come from `tune` where non-zero, else from
 *   the tuning cache entry for this batch (TRIOT_OP_BATCH, keyed by GPU, dtype, mode and
 *   the size classes floor(log2 n) and floor(log2 sum |y|); see triot_batch_autotune),
 *   else 1024 and 4; `tune` may be NULL.  Rejects descriptors whose x is not inside y,
 *   ranks out of range, NULL pointers or out-of-range tuning values (TRIOT_ERR_*;
 *   nothing is allocated then).
 */
int triot_batch_plan_create(const triot_batch_desc* descs, int n, int dtype, int mode,
                            const triot_tune* tune, triot_plan** out);
/*
 * triot_batch_run -- run the whole batch on `stream`.  The first run on a given stream
 *   captures the launch sequence into a CUDA graph; later runs replay it with one
 *   cudaGraphLaunch.  Pair buffers are read and written in place.
 */
int triot_batch_run(triot_plan* plan, void* stream);
/* Run the same work as plain per-pair launches (embed, product, moment per pair). */
int triot_batch_run_plain(triot_plan* plan, void* stream);
/* Bytes of device memory the plan holds, and its tile count. */
int triot_batch_plan_info(const triot_plan* plan, size_t* device_bytes, int64_t* tiles);
int triot_batch_plan_destroy(triot_plan* plan);
/* The geometry a plan runs with (threads per CTA, tile_elems, ctas_per_sm). */
int triot_batch_plan_geometry(const triot_plan* plan, triot_tune* out);
/*
 * triot_batch_autotune -- the batch's launch geometry chosen by measurement: for every
 *   candidate (tile_elems in {256, 512, 1024, 2048, 4096} x ctas_per_sm in {2, 4, 8}) a
 *   plan is built, run twice, then timed over three graph launches with CUDA events on
 *   `stream`; the fastest (median) is stored in the tuning cache under this batch's key
 *   (so that later triot_batch_plan_create calls with a NULL or zero `tune` use it, and
 *   triot_tune_save persists it) and returned in *best (may be NULL).  Runs the whole
 *   pipeline on the caller's buffers (each run rewrites every y and moment output the
 *   same way), allocates and frees candidate plans, and synchronises `stream`.  Errors as
 *   triot_batch_plan_create, or TRIOT_ERR_CUDA.
 */
int triot_batch_autotune(const triot_batch_desc* descs, int n, int dtype, int mode, void* stream,
                         triot_tune* best);

/* ------------------------------------------------------------------ tuning */

/* op codes for the tuning calls */
#define TRIOT_OP_EMBED 0
#define TRIOT_OP_CROP 1
#define TRIOT_OP_PRODUCT 2
#define TRIOT_OP_MOMENT 3
#define TRIOT_OP_BATCH 4   /* batches: see triot_batch_autotune */

/*
 * triot_autotune -- time candidate launch geometries for one (op, rank, shapes, dtype)
 *   on the caller's buffers (which it overwrites exactly as the op would) with CUDA
 *   events on `stream`, keep the fastest in the in-process cache (keyed by GPU, op,
 *   dtype, effective rank and inner-extent class) and return it in *best.  x and y are
 *   the op's own arguments in the op's order (TRIOT_OP_CROP writes x and reads y, despite
 *   the const on x here; embed and product write y).  For
 *   TRIOT_OP_MOMENT pass p as `x`, NULL as `y`, and a workspace large enough for every
 *   candidate (triot_moment_workspace_size with the largest geometry: use
 *   TRIOT_MOMENT_MAX_WORKSPACE_PER_RANK * (rank + 1) bytes).  Synchronises `stream`.
 */
#define TRIOT_MOMENT_MAX_WORKSPACE_PER_RANK (16384 * 8)
int triot_autotune(int op, int rank, const int64_t* xshape, const void* x,
                   const int64_t* yshape, void* y, int dtype, void* workspace,
                   size_t workspace_bytes, void* stream, triot_tune* best);
/* Read / force the cached geometry for the key of these arguments (no GPU work). */
int triot_tune_get(int op, int rank, const int64_t* xshape, const int64_t* yshape, int dtype,
                   triot_tune* out);
int triot_tune_set(int op, int rank, const int64_t* xshape, const int64_t* yshape, int dtype,
                   const triot_tune* tune);
/* Persist / restore the cache as JSON (one object per key).  Load merges entries. */
int triot_tune_save(const char* path);
int triot_tune_load(const char* path);
int triot_tune_clear(void);

/* ------------------------------------------------------------------ introspection */

/*
 * triot_canonicalize -- host only, no GPU work.  Shows how a call's shapes are reduced
 *   before launch: unit axes dropped (Section 4: trivial axes "can simply be ignored")
 *   and neighbouring axes merged where both tensors are contiguous across them (and, for
 *   embed, x is full along the inner one).  op: TRIOT_OP_EMBED / CROP / PRODUCT / MOMENT;
 *   yshape is ignored (may be NULL) for TRIOT_OP_MOMENT.  Writes the effective rank to
 *   *eff_rank and per effective axis (outermost first; arrays of TRIOT_MAX_RANK):
 *     ext     iteration extent (embed: y's, crop: x's, product: the intersection's,
 *             moment: p's),
 *     xstride x's stride in elements along the axis (moment: 0),
 *     ystride y's stride in elements (moment: 0),
 *     xbound  embed: x's extent along the axis (other ops: ext),
 *     orig    the first original axis merged into the axis (moment: its original axis).
 *   Any output pointer but eff_rank and ext may be NULL.
 */
int triot_canonicalize(int op, int rank, const int64_t* xshape, const int64_t* yshape,
                       int* eff_rank, int64_t* ext, int64_t* xstride, int64_t* ystride,
                       int64_t* xbound, int* orig);

/*
 * triot_fastdiv_check -- host only.  Runs the magic-multiplier division used by the
 *   kernels' flat-to-tuple decode (Granlund & Montgomery, "Division by invariant integers
 *   using multiplication", PLDI 1994) on `count` 32-bit dividends n[k] for divisor d
 *   (1 <= d < 2^31) and writes quotients q[k] and remainders r[k].  For tests.
 */
int triot_fastdiv_check(uint32_t d, const uint32_t* n, size_t count, uint32_t* q, uint32_t* r);

/*
 * triot_moment_plan -- which moment kernel triot_moment would launch for this shape and
 *   dtype under the tuning in force (no GPU work; needs the device's properties):
 *   *kernel = TRIOT_MK_ROWS (lane segments along the inner axis), TRIOT_MK_BLOCKS64 (f64
 *   block columns), TRIOT_MK_BLOCKS32 (float block columns), TRIOT_MK_WARPBLOCKS (float
 *   warp blocks) or TRIOT_MK_MARGINALS (rows x columns split: f64 tensors of at least 2^21
 *   elements, float tensors of at least 2^25 with 16-byte column runs), *grid = its CTAs
 *   (the partial vectors the combine adds), and for TRIOT_MK_MARGINALS *rows / *cols the
 *   matrix view (else 0).  Any output pointer may be NULL.
 */
#define TRIOT_MK_ROWS 0
#define TRIOT_MK_BLOCKS64 1
#define TRIOT_MK_BLOCKS32 2
#define TRIOT_MK_WARPBLOCKS 3
#define TRIOT_MK_MARGINALS 4
int triot_moment_plan(int rank, const int64_t* shape, int dtype, int* kernel, int* grid,
                      int64_t* rows, int64_t* cols);

/* Sticky device-side status (TRIOT_OK or TRIOT_ERR_DEVICE) of the current device; reading
 * it synchronises the device and clears it.  It is set when a kernel's bounded wait for a
 * staged copy gave up (the kernel then finishes with what it has, so its results are not
 * to be trusted) or when a batch work list holds a corrupted pair index. */
int triot_device_status(void);

/*
 * triot_selftest_wait_timeout -- a test of the failure path above, with nothing at risk:
 *   one warp waits on an mbarrier that expects an arrival nobody makes and that no copy
 *   targets, polling it `limit` times (1 .. 4096) with the same bounded wait the moment
 *   kernels use for their staged copies; the wait runs out, the kernel records it and
 *   returns.  The next triot_device_status() then returns TRIOT_ERR_DEVICE (and clears the
 *   flag); the context stays usable.  Not part of the paper's method.
 */
int triot_selftest_wait_timeout(int limit, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TRIOT_H */
