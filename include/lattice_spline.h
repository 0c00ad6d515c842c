/*
 * lattice_spline.h -- C ABI of the B300 lattice spline library.
 *
 * Evaluates f(x) = sum_{n in L Z^s} c_n phi(x - n) (Horacsek & Alim, Part II,
 * Eq. 1) for a piecewise-polynomial basis phi on a lattice L Z^s at many query
 * points, unrolled as in Algorithm 1: shift into the region of evaluation,
 * classify into a sub-region, fetch the coefficients of a fixed stencil and
 * evaluate the sub-region's polynomial.  A spline is described by the
 * sub-region table of Sec. 3 / Fig. 1; ls_spline_create generates a CUDA C++
 * kernel specialised to that table (the code generation of Sec. 4), compiles it
 * for sm_103a and loads it.
 *
 * Conventions shared by every entry point:
 *  - All device pointers are plain CUDA device addresses on the current device;
 *    all host pointers are ordinary host memory.  No call takes ownership of a
 *    caller buffer.  Library objects (ls_spline, ls_volume, ls_plan) are owned
 *    by the library and freed by their destroy call.
 *  - Points are FP32, row-major, dim values per point (x_0 fastest within a point).
 *  - A coefficient volume holds one array per Cartesian coset l_j of the
 *    storage grid scale*Z^dim: element (i_0, .., i_{dim-1}) of array j is the
 *    coefficient of site scale*i + l_j; all arrays have the same extent, axis 0
 *    fastest.  Three layouts (ls_layout): coset-major (array after array; the
 *    per-coset memory lookup of Sec. 4.1), coset-interleaved (the n_cosets
 *    values of one i adjacent) and bricked.  Sites outside the arrays
 *    contribute 0.
 *  - Calls that take a cudaStream_t are asynchronous on that stream (0 = the
 *    legacy default stream).  They return an ls_status describing argument
 *    validation and launch; a fault found by a kernel is not reported here.
 *  - No call aborts or traps; errors are returned as ls_status and a message
 *    readable with ls_last_error() (thread-local).
 */
#ifndef LATTICE_SPLINE_H
#define LATTICE_SPLINE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ls_spline_s *ls_spline;   /* generated + loaded kernels for one table */
typedef struct ls_volume_s *ls_volume;   /* coefficients of one spline on one grid   */
typedef struct ls_plan_s *ls_plan;       /* a batched persistent launch              */
typedef void *ls_stream;                 /* a cudaStream_t                           */

typedef enum {
    LS_OK = 0,
    LS_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad enum                 */
    LS_ERR_BAD_TABLE = 2,     /* inconsistent sub-region table                     */
    LS_ERR_UNSUPPORTED = 3,   /* valid but not supported (e.g. dim 1, > 64 sites)  */
    LS_ERR_OOM = 4,           /* device or host allocation failed                 */
    LS_ERR_CUDA = 5,          /* a CUDA runtime call failed (message has details)  */
    LS_ERR_COMPILE = 6,       /* NVRTC rejected the generated source              */
    LS_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up               */
    LS_ERR_DEVICE = 8         /* a kernel reported a fault in its status word      */
} ls_status;

typedef enum { LS_F32 = 0, LS_BF16 = 1, LS_F16 = 2, LS_F64 = 3 } ls_dtype;

/*
 * Memory layout of a coefficient volume with C cosets of P = prod(ext) values.
 * The value of coset j at grid index (i_0, i_1, i_2), q = i_0 + ext_0 (i_1 + ext_1 i_2), is
 *   LS_LAYOUT_COSET_MAJOR:  element j * P + q   (one array per coset, Sec. 4.1)
 *   LS_LAYOUT_INTERLEAVED:  element q * C + j   (cosets adjacent: the sites of
 *                           both BCC cosets, or of all four FCC cosets, near one
 *                           point share 32-byte sectors, so a stencil touches
 *                           fewer of them; identical to coset-major when C = 1)
 *   LS_LAYOUT_BRICKED:      element (b * V + w) * C + j, the grid cut into bricks
 *                           of 2 x 2 x 2 indices (2 x 2 in 2D; V = 8 or 4) in
 *                           x-fastest brick order b, w = (i_0 & 1) + 2 (i_1 & 1)
 *                           + 4 (i_2 & 1) inside the brick: with FP32 and two
 *                           cosets a 32-byte sector holds a 2 x 2 patch of both
 *                           cosets and a 128-byte line two bricks, so a compact
 *                           stencil touches fewer sectors and lines.  Needs even
 *                           extents and a spline created with ls_variant.brick = 1.
 *   LS_LAYOUT_BRICKED_SHIFTED: four bricked copies (3D, even extents): copy
 *                           c = s_0 + 2 s_1 (s in {0,1}^2) stores grid index i at
 *                           (i_0 + s_0, i_1 + s_1, i_2) of a bricked array over
 *                           extents (ext_0 + 2, ext_1 + 2, ext_2), element
 *                           c * Q + that array's bricked index, Q = C (ext_0 + 2)
 *                           (ext_1 + 2) ext_2; the padding is zero.  Each point's
 *                           gathers read the copy whose brick boundaries cut its
 *                           stencil into the fewest 32-byte sectors (a rule the
 *                           generator derives from the table; BCC quintic: 10.0
 *                           sectors per point instead of 11.3).  Read-only: the
 *                           evaluation kernels (value, gradient, Hessian, batched)
 *                           take it, the adjoint and the fit do not.  Needs a
 *                           spline created with ls_variant.brick = 2.
 *   LS_LAYOUT_BRICKED_SHIFTED_XYZ: the same with eight copies, the brick grid
 *                           also shifted on axis 2: copy c = s_0 + 2 s_1 + 4 s_2
 *                           over extents (ext_0 + 2, ext_1 + 2, ext_2 + 2).  For
 *                           the Cartesian splines, whose 32-byte sector is a whole
 *                           2 x 2 x 2 brick (tricubic: 8.0 sectors per point, the
 *                           least 64 sites can take).  ls_variant.brick = 3.
 */
typedef enum {
    LS_LAYOUT_COSET_MAJOR = 0,
    LS_LAYOUT_INTERLEAVED = 1,
    LS_LAYOUT_BRICKED = 2,
    LS_LAYOUT_BRICKED_SHIFTED = 3,
    LS_LAYOUT_BRICKED_SHIFTED_XYZ = 4
} ls_layout;

typedef enum {
    LS_ROE_PARALLELEPIPED = 0, /* k = floor(x) on the storage grid (Cartesian, scale 1)      */
    LS_ROE_VORONOI = 1         /* k = nearest lattice site (Voronoi cell of the lattice)     */
} ls_roe;

typedef enum {
    LS_FOLD_NONE = 0,          /* one sub-region: the whole region of evaluation             */
    LS_FOLD_SIGNED_PERM = 1    /* sub-regions are the images of y0 >= y1 >= .. >= 0 under the
                                  2^s s! signed permutations; T of Algorithm 1 is computed by
                                  sorting |y| instead of a table lookup                       */
} ls_fold;

/*
 * One reference sub-region (Fig. 1 table row without a transform; Algorithm 1,
 * psi_i).  On it, f(y) = sum_j c[k + T^T s_j] * w_j(T y - center), where k is the
 * shift into the region of evaluation, T the sub-region transform and
 *     w_j(u) = sum_a coef[j * n_monos + a] * prod_i u_i^{mono_exp[a * dim + i]}.
 * sites: n_sites * dim lattice offsets s_j (Cartesian, integer).
 */
typedef struct {
    int32_t n_sites;
    const int32_t *sites;
    int32_t n_monos;
    const int32_t *mono_exp;
    const double *coef;
    double center[3];
} ls_ref_region;

/*
 * Optional separable form of a tensor-product spline: along axis i,
 * w_j(u) = sum_a coef[j * (degree + 1) + a] u^a with u = y_i - center, for the
 * 1D sites sites[j]; the 3D weight of site (s_0, s_1, s_2) is the product.
 */
typedef struct {
    int32_t n_sites;
    const int32_t *sites;
    int32_t degree;
    const double *coef;
    double center;
} ls_axis_factor;

/*
 * Lattice + spline descriptor: a generator matrix, the coset offsets of the
 * storage grid and the sub-region table (Sec. 3, Algorithm 1).
 *   planes: n_planes * (dim + 1) doubles (p_i, d_i); bit i of q is set iff
 *           p_i . y - d_i >= 0 for the folded point y (Sec. 4.1, sub-region
 *           membership); the reference sub-region is sigma[q % bsp_mod].
 *   separable: NULL, or dim axis factors used instead of ref (LS_FOLD_NONE, the
 *           Cartesian grid L = I; the region of evaluation is [0,1)^dim for
 *           LS_ROE_PARALLELEPIPED or [-1/2,1/2]^dim around the nearest site for
 *           LS_ROE_VORONOI, and each factor one polynomial piece there).
 */
typedef struct {
    const char *name;                  /* nullable; [A-Za-z0-9_]{1,40}, used in kernel names */
    int32_t dim;                       /* 2 or 3 */
    int32_t roe;                       /* ls_roe */
    int32_t fold;                      /* ls_fold */
    int32_t scale;                     /* storage grid spacing (1 or 2) */
    double generator[9];               /* L, column-major (column j at [3j..3j+2]) */
    int32_t n_cosets;                  /* 1..8 */
    const int32_t *coset_offsets;      /* n_cosets * dim, each in [0, scale) */
    int32_t n_planes;                  /* 0..8 */
    const double *planes;
    int32_t bsp_mod;                   /* >= 1 */
    const int8_t *sigma;               /* bsp_mod entries, -1 = unused */
    int32_t n_ref;                     /* 1..15 */
    const ls_ref_region *ref;
    const ls_axis_factor *separable;
} ls_spline_desc;

/*
 * Kernel variants a spline can be generated with.  group / depth are the
 * group size m and pipeline depth d of Sec. 4.4 / Algorithm 2, counted in
 * stencil sites and groups: the gathers of group g are issued only after the
 * values of group g - depth have arrived (0 = no limit: all gathers at once).
 */
typedef struct {
    int32_t block;                     /* threads per block (default 256) */
    int32_t pts_per_thread;            /* T: consecutive points per thread; T > 1 reuses the gathers
                                          and coefficient transform while the region-of-evaluation
                                          site, fold and sub-region stay the same (ray order) */
    int32_t branchy;                   /* K > 1: 0 = evaluate all, select; 1 = branch */
    int32_t min_blocks;                /* __launch_bounds__ minimum blocks per SM (0 = none) */
    int32_t group;                     /* m: sites per gather group (0 = all) */
    int32_t depth;                     /* d: groups in flight (0 = unlimited) */
    int32_t blocks_per_sm;             /* grid = SMs x blocks_per_sm for the evaluation and the
                                          per-point adjoint kernels (0 = as many as fit); bounds
                                          the resident warps per SM without taking L1 away (no
                                          recompilation) */
    int32_t brick;                     /* 1: the kernels address LS_LAYOUT_BRICKED volumes (and only
                                          those); 2: LS_LAYOUT_BRICKED_SHIFTED volumes (3D); 3:
                                          LS_LAYOUT_BRICKED_SHIFTED_XYZ volumes (3D); 0: the linear
                                          layouts (coset-major, interleaved) */
    int32_t pipeline;                  /* 1: the value kernel issues the gathers of a thread's next
                                          point before evaluating the current one (software
                                          pipelining; non-separable tables; pts_per_thread ignored) */
    int32_t producers;                 /* P > 0: warp-specialized value kernel (non-separable tables):
                                          P producer warps per block gather the coefficients of 32
                                          points per consumer warp into shared memory, the other
                                          block / 32 - P warps evaluate the polynomials; bounded
                                          mbarrier waits (see ls_spline_status) */
    int32_t stage;                     /* S > 0: tile-staged value kernel for spatially sorted points
                                          (3D, LS_F32, linear layouts): a block bounds the sites of its
                                          blockDim consecutive points and, when they fit one tile of
                                          S^3 grid indices per coset (S = 1: 12 for the scale-2
                                          lattices, 16 for the Cartesian one; S must keep the tile's
                                          first row a multiple of 16 bytes), loads that tile with one
                                          TMA tensor copy and evaluates from shared memory; other
                                          blocks read global memory.  Results are bit-identical to
                                          the plain kernel.  Bounded mbarrier wait (ls_spline_status) */
    int32_t tensor;                    /* T > 0: the value kernel forms the coefficient transform
                                          A = M^T c of each tile of 128 points as one matrix product
                                          on the tensor cores (tcgen05.mma kind::tf32, three TF32
                                          products for FP32 accuracy, accumulator in tensor memory);
                                          one block per SM with S slots of 128 points: T = 1, as many
                                          as the 512 tensor-memory columns hold, at most 8 (at most 5
                                          for splines of K + N >= 64, whose registers fill the file);
                                          T = 2..8: T, at most what the columns hold; forces
                                          block = 128 S; non-separable tables.  Bounded mbarrier
                                          waits (ls_spline_status) */
    int32_t tensor_kind;               /* with tensor and FP32 coefficients: 0 = three TF32 products
                                          of the hi / lo split; 1 = three FP16 products: each point's
                                          coefficients scaled by a power of two (largest magnitude in
                                          [2^14, 2^15)), split into FP16 hi (11 significant bits) + lo
                                          (the rounded remainder), the scale undone on the results
                                          (half the tensor-memory columns per tile, so more tiles in
                                          flight).  Other values: LS_ERR_INVALID_ARG at create */
    int32_t plain_transform;           /* 1: the FMA kernels form each monomial coefficient A_a as the
                                          direct sum over the region's sites (one multiply-add per
                                          nonzero of the table); 0 (default): the generator factors the
                                          transform into sums and differences of site pairs (also of
                                          earlier sums) followed by a sparser table, wherever two rows
                                          of the table agree up to sign on enough monomials (the
                                          spline's symmetries make many do): the same A_a in fewer
                                          operations (BCC quintic 377 instead of 1016) */
    int32_t wait_limit;                /* bounded mbarrier waits (warp-specialized, staged and
                                          tensor-core kernels) give up after this many try_wait
                                          rounds (each suspends for at most about a microsecond) and
                                          set the status word (ls_spline_status); 0: 2^20 rounds */
    int32_t wait_probe;                /* failure-detection test hook, warp-specialized kernel only:
                                          1 = the producer warps never signal their slots, so every
                                          consumer wait runs out after wait_limit rounds and the
                                          kernel returns with the status word set and the outputs
                                          unwritten.  0 otherwise */
    int32_t prefetch;                  /* 1: each thread of the value and value + gradient kernels
                                          loads the coordinates of its next point before it
                                          evaluates the current one (FMA kernels) */
    int32_t l2_keep;                   /* 1: the value and value + gradient kernels load coefficients
                                          with an L2 evict-last cache policy (createpolicy), so the
                                          coefficient lines outlast the point and result streams,
                                          which are loaded and stored evict-first.  0 otherwise */
    int32_t fma2;                      /* 1: the factored coefficient transform forms pairs of monomial
                                          coefficients with paired FP32 FMA (fma.rn.f32x2), the constant
                                          pairs in __constant__ tables; same values (a variable only one
                                          of the pair reads adds an exact 0 to the other).  0 otherwise */
} ls_variant;

/* ---- status ---------------------------------------------------------------- */
const char *ls_status_str(ls_status s);
/* Message of the last failing call on this thread ("" if none). */
const char *ls_last_error(void);
/* Layout version of the structs above (8: ls_variant ends with fma2);
 * bindings compare it with their own before any other call. */
int32_t ls_abi_version(void);
/* Test hooks for failure detection (host-side injection; nothing faults on the
 * GPU).  ls_debug_fail_alloc(after): the library's next `after` device
 * allocations succeed and the one after them fails as if the device were out
 * of memory, so the call that makes it returns LS_ERR_OOM; after < 0 turns
 * the injection off (it is also off once it has fired).  The paper has no
 * counterpart.  ls_debug_live_allocs(): the device allocations the library
 * holds (volumes, status words, staging, plans, workspaces), for leak checks. */
void ls_debug_fail_alloc(int32_t after);
int64_t ls_debug_live_allocs(void);

/* ---- splines ----------------------------------------------------------------- */
/*
 * Validate the table, generate the specialised CUDA C++ (stencil and polynomials
 * unrolled, tables as immediates; Sec. 4.1-4.4), compile it with NVRTC for
 * sm_103a and load it on the current device.  coef_dtype selects the storage
 * type the kernels read (LS_F32, LS_BF16, LS_F16); arithmetic is FP32.
 * variant may be NULL (defaults).  Compiled cubins are cached on disk in the
 * directory named by LS_KERNEL_CACHE (default: a kcache/ folder beside the
 * library).  The descriptor is copied; the caller keeps ownership of it.
 * Errors: INVALID_ARG / BAD_TABLE / UNSUPPORTED / COMPILE / CUDA.
 */
ls_status ls_spline_create(const ls_spline_desc *desc, ls_dtype coef_dtype,
                           const ls_variant *variant, ls_spline *out);
ls_status ls_spline_destroy(ls_spline s);
/* Generate and compile into the on-disk cache only (no device needed): lets a
 * build step pay the NVRTC cost ahead of the first ls_spline_create. */
ls_status ls_spline_precompile(const ls_spline_desc *desc, ls_dtype coef_dtype,
                               const ls_variant *variant);
/* Generated source (NUL-terminated, owned by the spline) for inspection/tests. */
const char *ls_spline_source(ls_spline s);
/* The CUDA C++ source the generator emits for (desc, coef_dtype, variant),
 * without compiling it (host only, no device).  Copies at most cap bytes,
 * NUL-terminated, into buf (buf may be NULL with cap 0) and sets *len to the
 * source's length without the NUL, so a caller can size buf with a first call.
 * Errors: INVALID_ARG (len NULL) / BAD_TABLE / UNSUPPORTED. */
ls_status ls_spline_generate_source(const ls_spline_desc *desc, ls_dtype coef_dtype,
                                    const ls_variant *variant, char *buf, size_t cap, size_t *len);
/* LS_ERR_TIMEOUT if a bounded wait inside an evaluation kernel of this spline gave
 * up since the last call (the affected outputs are then incomplete), else LS_OK;
 * synchronises the stream and clears the word.  Only the warp-specialized value
 * kernel waits on anything. */
ls_status ls_spline_status(ls_spline s, ls_stream stream);
/* Counts the generator computed: stencil size (union over reference regions),
 * FP32 FMAs per point for f, for f + grad f, registers per thread of the eval kernel. */
ls_status ls_spline_info(ls_spline s, int32_t *n_sites, int32_t *fma_value,
                         int32_t *fma_grad, int32_t *regs_eval);

/* ---- coefficient volumes ----------------------------------------------------------- */
/*
 * A volume is a view of n_cosets coefficient arrays of extent ext[0..dim-1]
 * in the spline's coef_dtype, stored in `layout` (ls_layout).
 * ls_volume_create allocates them (library-owned, zero-filled); ls_volume_wrap
 * uses a caller device buffer of n_cosets * prod(ext) elements already in that
 * layout, which must outlive the volume.  Every kernel reads (and the adjoint
 * and the fit write) coefficients in the volume's layout.
 * Errors: INVALID_ARG (NULL, extent outside 1..2^20, unknown layout, a
 * bricked layout with extents that are not whole bricks, a layout the spline's
 * kernels do not address), UNSUPPORTED (2^31 or more coefficients), OOM.
 */
ls_status ls_volume_create(ls_spline s, const int64_t *ext, int32_t layout, ls_volume *out);
ls_status ls_volume_wrap(ls_spline s, const int64_t *ext, int32_t layout, void *device_coef,
                         ls_volume *out);
/* Copy (and convert) n_cosets*prod(ext) values of src_dtype from src (host or
 * device) into the volume.  src is in COSET-MAJOR layout; an interleaved
 * volume receives the values rearranged. */
ls_status ls_volume_upload(ls_volume v, const void *src, int32_t src_is_device,
                           ls_dtype src_dtype, ls_stream stream);
/* The volume's ls_layout (-1 for NULL). */
int32_t ls_volume_layout(ls_volume v);
/*
 * Copy n_cosets arrays of extent ext[0..dim-1] (ext[i] = 1 for i >= dim) with
 * elements of elem_bytes (2, 4 or 8) from src in src_layout to dst in
 * dst_layout (ls_layout): e.g. coefficients into the bricked layout, or an
 * adjoint result of an interleaved volume back to one array per coset.  src
 * and dst are distinct device buffers of n_cosets * prod(ext) elements.
 * Errors: INVALID_ARG (NULL or equal buffers, bad sizes, unknown layout, a
 * bricked side with extents that are not whole bricks).
 */
ls_status ls_relayout(const void *src, int32_t src_layout, void *dst, int32_t dst_layout,
                      int32_t n_cosets, const int64_t *ext, int32_t elem_bytes, ls_stream stream);
void *ls_volume_device_ptr(ls_volume v);
ls_status ls_volume_destroy(ls_volume v);

/* ---- evaluation (Algorithm 1) ----------------------------------------------------- */
/* out[i] = f(pts[i]) for i < n.  pts: n*dim device floats; out: n device floats. */
ls_status ls_eval(ls_volume v, const float *pts, int64_t n, float *out, ls_stream stream);
/*
 * f and its gradient from the differentiated sub-region polynomials (Sec. 3:
 * derivatives of the per-region polynomials, symmetry still applies):
 * grad[i*dim + d] = df/dx_d (pts[i]).  val may be NULL.
 */
ls_status ls_eval_grad(ls_volume v, const float *pts, int64_t n, float *val, float *grad,
                       ls_stream stream);
/*
 * f, its gradient and its Hessian from the twice-differentiated sub-region
 * polynomials (Sec. 3: derivatives of the per-region polynomials; the symmetry
 * transforms still apply: H = T^T H_ref T):
 * hess[i*6 + q] = d2f/dx_a dx_b (pts[i]) for (a,b) = (0,0) (1,1) (2,2) (0,1)
 * (0,2) (1,2) in 3D, hess[i*3 + q] for (0,0) (1,1) (0,1) in 2D.  val and grad may
 * be NULL.  Continuous for C^2 splines (tricubic, BCC quintic); elsewhere a
 * point on a knot plane gets the value of one of the adjacent polynomial pieces.
 */
ls_status ls_eval_hess(ls_volume v, const float *pts, int64_t n, float *val, float *grad, float *hess,
                       ls_stream stream);
/*
 * The linear texture fetch of Sec. 4.4.1 for 3D tensor-product splines with
 * FP32 coefficients in one array (trilinear, triquadratic, tricubic): pairs of
 * neighbouring sites become one hardware-interpolated fetch at the weighted
 * position, so at most 2 x 2 x 2 trilinear fetches replace the stencil's
 * gathers.  ls_volume_texture_sync copies the volume's current coefficients
 * into a texture (a 3D CUDA array owned by the volume, made on the first call;
 * zero outside the arrays); call it again after changing them.
 * ls_eval_linear_fetch evaluates from that copy: out[i] = f(pts[i]) within
 * 6/256 ||c||_inf, because the texture unit interpolates with 8-bit fixed-point
 * fractions (not for the 2e-6 accuracy of ls_eval).
 * Errors: UNSUPPORTED (not such a spline or storage), INVALID_ARG (not synced).
 */
ls_status ls_volume_texture_sync(ls_volume v, ls_stream stream);
ls_status ls_eval_linear_fetch(ls_volume v, const float *pts, int64_t n, float *out, ls_stream stream);
/*
 * Same as ls_eval with HOST buffers: copies pts to the device, evaluates and
 * copies out back; returns when out is complete.  The points move in chunks
 * on two internal streams, so the host-to-device copy of one chunk, the kernels
 * of another and the device-to-host copy of a third overlap.  Pinned host
 * memory gives asynchronous copies; pageable memory works but serialises.
 * Work is ordered after everything already queued on `stream`.  Staging
 * buffers and the two streams belong to the volume (made on first use).
 */
ls_status ls_eval_host(ls_volume v, const float *host_pts, int64_t n, float *host_out,
                       ls_stream stream);
/*
 * ls_eval_host for n_vol volumes (same dimension) at the same host points: the
 * points cross to the device once, every volume is evaluated per chunk, and
 * host_out[k] receives the values of vols[k].  Staging belongs to vols[0].
 */
ls_status ls_eval_host_multi(int32_t n_vol, const ls_volume *vols, const float *host_pts, int64_t n,
                             float *const *host_out, ls_stream stream);

/*
 * How ls_adjoint_coef sums the contributions of the points to a coefficient.
 *   LS_ADJ_ATOMIC:        one FP32 atomicAdd per (point, stencil site); the
 *                         result depends on the order in its last bits.
 *   LS_ADJ_DETERMINISTIC: the points are binned by their region-of-evaluation
 *                         site and every coefficient sums its contributions in
 *                         a fixed order: bitwise reproducible (needs scratch).
 *   LS_ADJ_ATOMIC_WARP:   as LS_ADJ_ATOMIC, but the lanes of a warp that hit the
 *                         same coefficient first add their values by shuffles
 *                         (__match_any_sync) and one of them issues the atomic:
 *                         fewer atomics when neighbouring points share sites
 *                         (Morton-sorted or ray-ordered points).
 *   LS_ADJ_DETERMINISTIC_FIXED: every value g * w is rounded to a multiple of
 *                         2^-s and added exactly in an int64 per coefficient
 *                         (integer atomics, so the order does not matter), then
 *                         converted once: bitwise reproducible at about the
 *                         atomic speed (needs scratch).  2^s is the largest
 *                         power of two with sum|gout| * wmax * 2^s < 2^61
 *                         (wmax: a bound on |phi| the generator derives from the
 *                         table), so no sum can overflow; each value is off by at
 *                         most 2^-(s+1) before the final FP32 rounding.  A
 *                         non-finite gout gives an unspecified result.
 *   LS_ADJ_ATOMIC_TILED:  for spatially sorted points (Morton order): a block
 *                         of consecutive points whose stencils fit one tile of
 *                         grid indices (edge up to 16 on BCC/FCC, 24 on the
 *                         Cartesian grid, at most 48 KiB of shared memory;
 *                         variant.stage > 1 sets the edge)
 *                         sums its contributions in shared memory and adds
 *                         each touched coefficient to dcoef once; other blocks
 *                         add per (point, site) as LS_ADJ_ATOMIC.  Order-
 *                         dependent in the last bits, like LS_ADJ_ATOMIC.
 *   LS_ADJ_DETERMINISTIC_FIXED_TILED: the same tiling on the fixed-point
 *                         integers of LS_ADJ_DETERMINISTIC_FIXED: bitwise
 *                         identical to that mode (needs its scratch).
 * The tiled modes need a linear layout (coset-major or interleaved); on a
 * bricked volume they run as their untiled counterparts.
 */
typedef enum {
    LS_ADJ_ATOMIC = 0,
    LS_ADJ_DETERMINISTIC = 1,
    LS_ADJ_ATOMIC_WARP = 2,
    LS_ADJ_DETERMINISTIC_FIXED = 3,
    LS_ADJ_ATOMIC_TILED = 4,
    LS_ADJ_DETERMINISTIC_FIXED_TILED = 5
} ls_adjoint_mode;

/*
 * Adjoint with respect to the coefficients (transposed stencil):
 *     dcoef[site n] += sum_i gout[i] * phi(pts[i] - n)
 * The derivative of Eq. 1 with respect to c_n; not part of the paper, which
 * only evaluates f.  dcoef: FP32 device array with the volume's layout
 * (n_cosets * prod(ext)), accumulated into.  mode: ls_adjoint_mode.
 * scratch (the two deterministic modes only): device buffer of at least
 * ls_adjoint_scratch_bytes(v, n) bytes (NULL: the call allocates and frees it).
 * Errors: INVALID_ARG (NULL buffers, n < 0, unknown mode), OOM, UNSUPPORTED
 * (deterministic mode with 2^31 or more points or bins).
 */
ls_status ls_adjoint_coef(ls_volume v, const float *pts, const float *gout, int64_t n,
                          float *dcoef, int32_t mode, void *scratch,
                          ls_stream stream);
size_t ls_adjoint_scratch_bytes(ls_volume v, int64_t n);

/* ---- Morton order of points -------------------------------------------------------- */
/*
 * perm[0..n) = indices of pts ordered by the 30-bit Morton code of the cell
 * floor((x - origin) / cell) (10 bits per axis, clamped to [0, 1023]); ties keep
 * input order (stable LSD radix sort).  keys_out (nullable) receives the sorted keys.
 * scratch: device buffer of ls_morton_scratch_bytes(n) bytes (NULL: allocated).
 */
ls_status ls_morton_sort(const float *pts, int64_t n, const float *origin, float cell,
                         int32_t *perm, uint32_t *keys_out, void *scratch, ls_stream stream);
size_t ls_morton_scratch_bytes(int64_t n);
/*
 * ls_morton_sort without any device allocation (the paper has no counterpart).
 * Same arguments and results as ls_morton_sort with scratch = NULL, for
 * callers that must not allocate device memory while they run (a framework
 * whose caching allocator owns the device memory, a latency-bound loop that
 * cannot absorb cudaMalloc/cudaFree, a fixed up-front memory budget).  Its
 * scratch is one static 3.75 MiB device array compiled into the library, which
 * every GPU that loads the library holds until the process exits.
 *  - n is limited to 262144 (2^18) points; larger n returns LS_ERR_INVALID_ARG
 *    with a message.  It calls no cudaMalloc, cudaFree or allocating routine.
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (with that device current); make that first call
 *    before any stream capture.  Under CUDA's lazy module loading that first
 *    call (its symbol lookup and first kernel launches) may also load the
 *    library's modules onto the device, which takes device memory once; the
 *    no-allocation guarantee holds from the second call on a device.
 *  - All calls share the one array and it keeps the last call's contents;
 *    nothing in it has to start at zero.  Calls whose work overlaps on the GPU
 *    (other streams, other threads, same device) race on it: serialise them.
 */
ls_status ls_morton_sort_noalloc(const float *pts, int64_t n, const float *origin, float cell,
                                 int32_t *perm, uint32_t *keys_out, ls_stream stream);
/* dst[i] = src[perm[i]] for rows of `width` floats (gather), or the inverse scatter. */
ls_status ls_permute_rows(const float *src, const int32_t *perm, int64_t n, int32_t width,
                          int32_t inverse, float *dst, ls_stream stream);

/*
 * Measurement probe for the gather roofline: every one of nthreads threads
 * issues loads_per_thread independent 4-byte loads from table at hashed indices
 * in [0, 2^floor(log2(table_elems))) and writes their sum to out[thread].
 * blocks: grid size (0 = 148 * 8).
 */
ls_status ls_probe_gather(const float *table, int64_t table_elems, int32_t loads_per_thread, float *out,
                          int64_t nthreads, int32_t blocks, ls_stream stream);

/* ---- batched persistent evaluation ------------------------------------------------ */
/*
 * One plan evaluates n_vol volumes (any mix of splines whose kernels were
 * generated in the same ls_plan_create), each at its own point batch, in ONE
 * persistent launch: blocks pull (volume, tile) items from a device work list.
 * pts[v], out[v]: device pointers; n[v]: point counts.  The plan copies the
 * arrays; the buffers must stay valid while the plan is launched.
 * ls_plan_launch only enqueues one kernel (no allocation, no host sync) and may
 * be captured into a CUDA graph.  tile: points per work item; 0 = autotuned: ls_plan_create
 * then times the kernel for several tile sizes (launching it on the volumes' data) and
 * keeps the fastest; results are cached per (kernel, volume sizes) for the process.
 */
ls_status ls_plan_create(int32_t n_vol, const ls_volume *vols, const float *const *pts,
                         const int64_t *n, float *const *out, int32_t tile, ls_plan *plan);
/* The tile (points per work item) the plan uses, and the block size of its kernel. */
ls_status ls_plan_info(ls_plan plan, int32_t *tile, int32_t *block, int32_t *n_items, int32_t *grid);
ls_status ls_plan_launch(ls_plan plan, ls_stream stream);
/* Status word of the launches so far (LS_OK, or LS_ERR_DEVICE if a work item named an
 * unknown spline); synchronises the stream.  The persistent kernel never waits: blocks
 * take items with an atomic ticket until the list is exhausted. */
ls_status ls_plan_status(ls_plan plan, ls_stream stream);
ls_status ls_plan_destroy(ls_plan plan);

/* ---- least-squares fit -------------------------------------------------------------- */
/*
 * Fit coefficients c to samples y_i at pts_i by CGLS on
 *     min_c ||A c - y||^2 + lambda ||c||^2,   A[i, n] = phi(pts_i - n),
 * with A c from ls_eval and A^T r from ls_adjoint_coef in adjoint_mode
 * (ls_adjoint_mode; LS_ADJ_DETERMINISTIC makes the whole fit bitwise reproducible).  Dot products and norms are FP64 on the device.  coef
 * (the volume's FP32 array) holds the initial guess and receives the result.
 * Stops after max_iter iterations or when ||A^T r|| <= rel_tol ||A^T y||.
 * resid_hist (host, nullable, max_iter + 1 doubles): ||A^T r||_2 per iteration.
 * iters (host, nullable): iterations done.
 */
ls_status ls_cg_fit(ls_volume v, const float *pts, const float *y, int64_t n, double lambda,
                    int32_t max_iter, double rel_tol, int32_t adjoint_mode,
                    double *resid_hist, int32_t *iters, ls_stream stream);

/* ---- device helpers used by the FP64 parts of the fit -------------------------------- */
/* *result (device double) = sum_i a[i] * b[i] accumulated in FP64. */
ls_status ls_dot_f64(const float *a, const float *b, int64_t n, double *result, ls_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* LATTICE_SPLINE_H */
