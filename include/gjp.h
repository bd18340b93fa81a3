/*
 * gjp.h -- C ABI of the GB300 (sm_103a) branchless generalized Joseph
 * projector (GJP): cone-beam forward projection of a voxel volume and its
 * matched adjoint.
 *
 * Method: J. Graetz, "High performance volume ray casting: A branchless
 * generalized Joseph projector" -- Algorithm 1 with Eq. 1-13.  For every
 * detector pixel of every view the source-to-pixel ray is marched plane by
 * plane along its dominant ("driving") axis m (Eq. 3), sampled at the
 * integer planes p_m = 0 .. n_m - 1 (Eq. 5-6), the volume is interpolated
 * bilinearly among the four neighbours in each plane (Eq. 7-12, w_lin of
 * Eq. 13) and the samples are summed with the path-length weight |rt|
 * (Algorithm 1) -- here |h (.) rt|, the world length of one plane step for
 * voxel size h.  Taps outside the grid read zero.
 *
 * Conventions shared by every entry point
 *  - Volume: C-contiguous [nx][ny][nz] (z fastest), voxel (i,j,k) centred at
 *    world origin + (i*hx, j*hy, k*hz).  origin == NULL means the centred
 *    grid, origin_k = -(n_k - 1)/2 * h_k.
 *  - Projections: C-contiguous float32 [n_views][nv][nu] (iu fastest).
 *    Pixel (iu, iv) of view k is centred at
 *    det_origin[k] + iu*det_u[k] + iv*det_v[k]  (world units).
 *  - Output unit: world length x volume value.
 *  - Device pointers are caller-owned CUDA device memory on the current
 *    device; the library never frees them.  `stream` is a cudaStream_t
 *    (NULL = legacy default stream).  Calls are stream-ordered and
 *    asynchronous; nothing synchronises the host.
 *  - Errors are returned, never raised (no abort/exit/trap).  A kernel
 *    failure that is only detected asynchronously surfaces from the CUDA
 *    runtime on a later synchronisation, as for any CUDA library.
 *  - The first call for a given (geometry, device, volume grid) builds and
 *    uploads a per-view table (a few dozen bytes per view, allocated with
 *    cudaMalloc and owned by the geometry).  Make that first call before
 *    capturing a stream into a CUDA graph; later calls only launch kernels.
 */
#ifndef GJP_H
#define GJP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GJP_OK = 0,
    GJP_ERR_INVALID_ARG = 1, /* a pointer, size or geometry value is rejected */
    GJP_ERR_UNSUPPORTED = 2, /* valid but not implemented (e.g. dtype for adjoint) */
    GJP_ERR_OOM = 3,         /* host or device allocation failed */
    GJP_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    GJP_ERR_INTERNAL = 5,
    GJP_ERR_TIMEOUT = 6
} gjp_status;

/* Storage type of the volume read by gjp_forward.  16-bit volumes are
 * widened to float32 on load; interpolation weights and accumulation are
 * float32 for every storage type. */
typedef enum { GJP_F32 = 0, GJP_BF16 = 1, GJP_F16 = 2 } gjp_dtype;

/* Opaque, library-owned projection geometry. */
typedef struct gjp_geometry gjp_geometry;

/*
 * gjp_geometry_create -- describe n_views flat-panel cone-beam views (the
 * source point s and pixel locations d that define the rays of Algorithm 1,
 * Eq. 1-2).
 *   src, det_origin, det_u, det_v : host arrays [n_views][3] of doubles in
 *       world units (source position; centre of pixel (0,0); displacement
 *       per +1 in iu; displacement per +1 in iv).  They are copied; the
 *       caller keeps ownership.
 *   nu, nv : detector columns (iu) and rows (iv), >= 1.
 *   out    : receives the new geometry (set to NULL on error).
 * Returns GJP_ERR_INVALID_ARG for n_views < 1, nu/nv < 1, NULL pointers,
 * non-finite values, a zero or parallel det_u/det_v, or a source lying in
 * its detector plane (which would allow a zero-length ray).  Host only: no
 * CUDA call is made.
 */
gjp_status gjp_geometry_create(int n_views, int nu, int nv, const double *src,
                               const double *det_origin, const double *det_u,
                               const double *det_v, gjp_geometry **out);

/* Frees the geometry and its device tables (NULL-safe).  Device tables are
 * freed with cudaFree, which waits for work that may still use them. */
void gjp_geometry_destroy(gjp_geometry *g);

/* Interpolation weight function w(d) of Eq. 9-12: GJP_WEIGHT_LIN is
 * w_lin(d) = 1 - d (Eq. 13, multilinear, the default); GJP_WEIGHT_SPL is
 * w_spl(d) = 1 - 3d^2 + 2d^3 (Eq. 14, C1 at the grid points). */
typedef enum { GJP_WEIGHT_LIN = 0, GJP_WEIGHT_SPL = 1 } gjp_weight;

/* Selects the weight function used by every later projection with g
 * (forward and adjoint alike, so the pair stays transposed).  The GATHER
 * families support both weights; SLAB and PREFETCH implement w_lin only and
 * return GJP_ERR_UNSUPPORTED when asked for with w_spl (AUTO then uses
 * GATHER).  Returns GJP_ERR_INVALID_ARG for NULL or an unknown weight. */
gjp_status gjp_geometry_set_weight(gjp_geometry *g, gjp_weight w);

/*
 * gjp_geometry_set_launch -- launch shape of the one-thread-per-ray kernels
 * (gather forward, prefetch forward, gather adjoint, footprint) for every
 * later call with g.  It changes only how work is laid out on the GPU, never
 * a result: each ray is still marched by one thread with the same
 * arithmetic.  The paper tunes the CUDA block size per configuration; this
 * is that knob, plus the order in which blocks are issued.
 *   tile_u     : detector columns per block, 1, 2, 4 (default) or 8; a
 *                block is tile_u warps of 32 detector rows.
 *   view_group : 1 .. 64.  Blocks are issued so that view_group
 *                consecutive views are processed tile by tile together
 *                (their rays cross nearly the same voxels, which then come
 *                from the L2 cache); 1 issues the views one after another.
 *                Until this call is made, each launch picks it from the
 *                grid and the scan: a group spans 16 degrees of rotation
 *                at 512 voxels per edge, scaled by (512 / longest edge)^2,
 *                divided by the median angle between consecutive views'
 *                central rays and held to 1 .. 16 views (wider groups
 *                would outgrow the L2); gjp_geometry_get_launch then
 *                reports 16.
 * Returns GJP_ERR_INVALID_ARG for NULL or a value outside those sets.
 */
gjp_status gjp_geometry_set_launch(gjp_geometry *g, int tile_u, int view_group);

/*
 * gjp_geometry_set_fov -- field-of-view cylinder of the paper's speed
 * section, where the first sampling point and the number of samples of
 * each ray follow its intersection with a cylindrical volume rather than
 * with the bounding box.  With radius > 0 (world units) every later
 * projection with g -- forward families, adjoints, batches, footprints --
 * samples a ray only on the planes whose sample lies within `radius` of the
 * line through the volume centre parallel to z (the rotation axis of a
 * centred circular scan); 0 (the default) turns it off.  The adjoint skips
 * the same samples, so it stays the transpose.  For a volume that is zero
 * farther than radius - 2 voxels from that line the result equals the
 * unclipped one (up to float32 rounding) with fewer samples; for other
 * volumes it is the projection of the volume cut to the cylinder, with the
 * plane decision made in float32 (a sample within ~1e-4 voxel of the
 * cylinder wall may fall on either side).  Returns GJP_ERR_INVALID_ARG for
 * NULL, a negative or a non-finite radius.
 */
gjp_status gjp_geometry_set_fov(gjp_geometry *g, double radius);

/* Reads back the launch shape set by gjp_geometry_set_launch (or the
 * library defaults).  Either output pointer may be NULL. */
gjp_status gjp_geometry_get_launch(const gjp_geometry *g, int *tile_u, int *view_group);

/* Reads back the detector shape of a geometry.  Any output pointer may be NULL. */
gjp_status gjp_geometry_info(const gjp_geometry *g, int *n_views, int *nu, int *nv);

/*
 * gjp_forward -- GJP line integrals (Algorithm 1) of every pixel of every
 * view of g through the volume.
 *   d_volume : device, [nx][ny][nz] elements of `dtype` (2- or 4-byte
 *              aligned as the type requires).
 *   voxel_size : host double[3] (hx, hy, hz) > 0.
 *   volume_origin : host double[3] world centre of voxel (0,0,0), or NULL.
 *   d_proj   : device float32 [n_views][nv][nu]; fully overwritten.
 * Returns GJP_ERR_INVALID_ARG for NULL pointers, sizes < 1, bad voxel size,
 * an unknown dtype, or a source inside the volume's bounding box (the
 * method integrates the whole line through the volume, which assumes
 * source and detector outside it).
 */
gjp_status gjp_forward(const void *d_volume, gjp_dtype dtype, int64_t nx, int64_t ny, int64_t nz,
                       const double voxel_size[3], const double volume_origin[3],
                       const gjp_geometry *g, float *d_proj, void *stream);

/* Kernel family used by gjp_forward_ex. */
typedef enum {
    GJP_PATH_AUTO = 0,   /* the library's fastest family for the call (forward: PAIRS for
                            16-bit storage over 32 or more views and 2^27 view-voxels
                            where it applies, else GATHER; adjoint: COMBINE) */
    GJP_PATH_GATHER = 1, /* one thread per ray, taps gathered from global memory */
    GJP_PATH_SLAB = 2,   /* detector tiles stream per-plane voxel boxes into shared memory
                            with TMA; needs a 16-byte aligned volume whose z row is a
                            multiple of 16 bytes and a magnification the box sizes cover */
    GJP_PATH_PREFETCH = 3, /* gather, with each warp's footprint a few planes ahead
                            prefetched into L2 by TMA; same volume alignment as SLAB */
    GJP_PATH_COMBINE = 4, /* adjoint only: neighbouring rays of a warp hand shared taps to
                            one another before the atomic additions (see gjp_adjoint_ex) */
    GJP_PATH_TEXTURE = 5, /* forward only, float32 / float16 volumes: the four taps of a
                            sample come from one texture gather (tld4) on a layered copy of
                            the volume; exact float32 weights (see below) */
    GJP_PATH_HWLIN = 6,   /* forward only, float32 / float16 volumes, w_lin: GJP_hwlin, one
                            hardware-filtered 3-D texture fetch per sample; the hardware
                            quantises the interpolation weights to 1/256 (see below) */
    GJP_PATH_PAIRS = 7    /* forward only: GATHER, with the row-table march reading a
                            z-paired copy of the volume (see below) */
} gjp_path;

/*
 * gjp_forward_ex -- gjp_forward with an explicit kernel family.  GATHER,
 * SLAB, PREFETCH and TEXTURE compute the same samples with the same
 * arithmetic (results agree to float32 rounding).  GJP_PATH_SLAB returns
 * GJP_ERR_UNSUPPORTED when its conditions are not met; GJP_PATH_AUTO never
 * does.
 *
 * The texture families (the texture-memory and hardware-interpolation
 * variants of the paper's speed section) copy the volume on every call into
 * texture arrays that the library allocates on first use and keeps with the
 * geometry until gjp_geometry_destroy: two layered arrays (TEXTURE; twice
 * the volume's size) or one 3-D array (HWLIN; once the volume's size).
 * Texture border addressing supplies the zero border.  They return
 * GJP_ERR_UNSUPPORTED for bfloat16 volumes (no such texture format), for a
 * grid beyond the device's texture limits, and (HWLIN) for w_spl; calls of
 * a texture family with the same geometry and grid must not overlap on the
 * GPU (they share the arrays).  HWLIN's 1/256 weight steps put its error
 * near 1e-4 .. 1e-3 of the projection maximum: above the float32 parity
 * bound, so GJP_PATH_AUTO never takes it.
 *
 * PAIRS first writes a z-paired copy of the volume, whose element e holds
 * voxels e and e + 1 of the same z line (the upper one zero past the last
 * z), and the row-table march of GATHER then reads both z taps of a row with
 * one aligned load (8 bytes for float32, 4 for 16-bit storage) instead of
 * two; every other part of GATHER is unchanged and the results are bitwise
 * equal to GATHER's.  The copy (8 or 4 bytes per voxel) is allocated on
 * `stream` from a memory pool of the library and released on `stream`
 * after the projection; the pool keeps up to 8 GiB for later calls (see
 * gjp_trim_workspace).  PAIRS returns GJP_ERR_UNSUPPORTED while `stream`
 * is being captured into a CUDA graph and for grids whose element offsets
 * do not fit 32 bits, and GJP_ERR_OOM when the copy cannot be allocated.
 * GJP_PATH_AUTO takes PAIRS for bfloat16 and float16 storage when g has at
 * least 32 views and views x voxels is at least 2^27 (measured faster than
 * GATHER there: half the load instructions, same L1 lines per load; with
 * fewer views the volume is read from DRAM about once and the copy only
 * adds bytes, and below that work the copy is not repaid) and falls back to
 * GATHER wherever PAIRS returns one of those statuses; for float32 it takes
 * GATHER (the 8-byte copy doubles the footprint in the caches and measured
 * slower).
 */
gjp_status gjp_forward_ex(const void *d_volume, gjp_dtype dtype, int64_t nx, int64_t ny, int64_t nz,
                          const double voxel_size[3], const double volume_origin[3],
                          const gjp_geometry *g, float *d_proj, gjp_path path, void *stream);

/*
 * gjp_stream_status -- synchronises `stream` and reports whether any kernel
 * of this library gave up a bounded wait since the last call
 * (GJP_ERR_TIMEOUT; the flag is then cleared).  Such a kernel returns
 * without hanging the device but its output is not valid.  A library built
 * with GJP_CHECK_TAPS=1 also reports GJP_ERR_INTERNAL (taking precedence)
 * when a kernel met a tap outside the grid in a plane range it marches
 * without per-tap tests (see gjp_selftest_tap_check).
 */
gjp_status gjp_stream_status(void *stream);

/*
 * gjp_selftest_wait_timeout -- failure-detection self-test (the paper has
 * no counterpart): launches on `stream` one kernel whose thread waits,
 * through the same bounded wait as the library's pipelines, on a barrier
 * phase that nothing ever completes.  The wait gives up after its limit
 * (one second of wall time), the kernel records the timeout and returns,
 * and the next gjp_stream_status(stream) reports GJP_ERR_TIMEOUT; the GPU
 * context stays usable.  Touches no caller memory.
 */
gjp_status gjp_selftest_wait_timeout(void *stream);

/*
 * gjp_selftest_tap_check -- self-test of the debug build (the paper has no
 * counterpart).  A library compiled with GJP_CHECK_TAPS=1 range-checks every
 * tap that the interior plane marches (Algorithm 1's loop over the planes
 * whose four Eq. 12 taps all lie in the grid) read or reduce without a
 * per-tap test: a tap outside the grid is skipped, not accessed, and
 * recorded, and the next gjp_stream_status reports GJP_ERR_INTERNAL (once;
 * the record is cleared).  This call queues on `stream` one thread that
 * records such a tap through the same check, touching no memory, so that a
 * test can see the report path work.  Returns GJP_ERR_UNSUPPORTED in the
 * production build, which has no check.
 */
gjp_status gjp_selftest_tap_check(void *stream);

/*
 * gjp_debug_fail_allocations -- failure-injection hook for tests (the paper
 * has no counterpart): the next `n` device allocations that the library
 * attempts (per-view tables, batch queues, texture arrays, z-paired
 * copies) fail as if the device were out of memory, so the calls that need
 * them return GJP_ERR_OOM and leave their outputs untouched (GJP_PATH_AUTO
 * reads the volume directly instead of a z-paired copy it could not
 * allocate); later allocations proceed.
 * n = 0 clears it.  Host-only, thread-safe; no GPU fault is involved.
 * Returns GJP_ERR_INVALID_ARG for n < 0.
 */
gjp_status gjp_debug_fail_allocations(int n);

/*
 * gjp_trim_workspace -- returns to the device the memory that the
 * library's workspace pools keep between calls (the z-paired copies of
 * GJP_PATH_PAIRS; up to 8 GiB per device).  Waits for nothing: memory that
 * a queued call still uses is kept until that call is done.  Safe to call
 * at any time; GJP_OK unless CUDA reports an error.
 */
gjp_status gjp_trim_workspace(void);

/*
 * gjp_adjoint -- matched transpose of gjp_forward (float32 volume):
 * d_volume (+)= A^T d_proj, where A is the system matrix of gjp_forward
 * (the g = A f view of the reconstruction section).  Every (ray, plane,
 * tap) triple of the forward pass scatters proj * |h (.) rt| * weight into
 * its voxel, so <A x, y> = <x, A^T y> up to float32 rounding.
 *   d_proj   : device float32 [n_views][nv][nu].
 *   d_volume : device float32 [nx][ny][nz]; zeroed first unless
 *              `accumulate` is non-zero.
 * The scatter uses float32 atomic additions, so the summation order (and
 * the last bits of the result) can differ between runs.
 * Errors as for gjp_forward.
 */
gjp_status gjp_adjoint(const float *d_proj, const gjp_geometry *g, int64_t nx, int64_t ny,
                       int64_t nz, const double voxel_size[3], const double volume_origin[3],
                       float *d_volume, int accumulate, void *stream);

/*
 * gjp_adjoint_ex -- gjp_adjoint with an explicit kernel family:
 * GJP_PATH_GATHER scatters every tap with a float32 atomic addition to
 * global memory; GJP_PATH_SLAB accumulates each detector tile's taps for a
 * few planes in shared memory and adds the whole box to the volume with one
 * TMA bulk tensor reduction (same volume alignment conditions as the slab
 * forward; tiles with mixed driving axes fall back to the scatter);
 * GJP_PATH_COMBINE lets each warp whose 32 rays share their transverse row
 * (a circular orbit about z with detector rows along z) march its planes in
 * step and hand each ray's upper z tap to the neighbouring ray that has the
 * same voxel as its lower tap, so one atomic addition carries both (half
 * the additions); other warps scatter tap by tap.  GJP_PATH_AUTO takes
 * COMBINE.  GJP_PATH_PREFETCH is not an adjoint family
 * (GJP_ERR_INVALID_ARG).  Results agree to float32 rounding; none is
 * bitwise deterministic.
 */
gjp_status gjp_adjoint_ex(const float *d_proj, const gjp_geometry *g, int64_t nx, int64_t ny,
                          int64_t nz, const double voxel_size[3], const double volume_origin[3],
                          float *d_volume, int accumulate, gjp_path path, void *stream);

/*
 * gjp_footprint -- measurement helper (not part of the method): sets
 * d_marks[voxel] = 1 for every voxel that receives a non-zero
 * interpolation weight from some ray of view `view` (the view's compulsory
 * volume traffic, used for roofline accounting).  d_marks is device memory
 * of nx*ny*nz bytes, zeroed by the caller; other bytes are left unchanged.
 * Errors as for gjp_forward, plus GJP_ERR_INVALID_ARG for a view index
 * outside [0, n_views).
 */
gjp_status gjp_footprint(const gjp_geometry *g, int view, int64_t nx, int64_t ny, int64_t nz,
                         const double voxel_size[3], const double volume_origin[3],
                         unsigned char *d_marks, void *stream);

/*
 * gjp_forward_noalloc -- gjp_forward that allocates no memory.  The paper
 * has no counterpart of this entry point; it exists for callers that cannot
 * let a library allocate device memory once they are running: a framework
 * that hands a fixed device-memory budget to its components, a real-time
 * reconstruction loop that forbids allocation after acquisition starts, or a
 * plug-in that must not touch its host application's allocator.
 *
 * It computes exactly what gjp_forward computes (the same per-view table
 * and the same gather kernels, so the projections are bitwise equal; it
 * always reads the volume itself, never a z-paired copy, whose taps are
 * the same values), but
 * keeps the per-view table in a fixed array of GJP_NOALLOC_MAX_VIEWS entries
 * (144 bytes each, about 144 KiB) that the CUDA runtime places on every GPU
 * that loads this library and keeps there until the process exits.  The
 * table is formed on the host and written into that array on `stream`,
 * ahead of the projection, by a small copy kernel that receives up to 64
 * views per launch as its by-value parameters; the call performs no
 * cudaMalloc, cudaFree, host-to-device memcpy or other allocation, and
 * returns without waiting for the GPU.
 *   - Geometries with more than GJP_NOALLOC_MAX_VIEWS views are rejected
 *     with GJP_ERR_UNSUPPORTED (split the views over several calls).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current).  Make that first
 *     call before capturing a stream into a CUDA graph.
 *   - All calls on a device share the one array and each overwrites it; it
 *     keeps the last call's table.  Calls that may overlap on the GPU (on
 *     different streams, or from different host threads) race on it: order
 *     them on one stream or synchronise between them.  Nothing in the array
 *     needs to start at zero.
 * Arguments, layouts and other errors as for gjp_forward.
 */
#define GJP_NOALLOC_MAX_VIEWS 1024
gjp_status gjp_forward_noalloc(const void *d_volume, gjp_dtype dtype, int64_t nx, int64_t ny, int64_t nz,
                               const double voxel_size[3], const double volume_origin[3],
                               const gjp_geometry *g, float *d_proj, void *stream);

/*
 * Batched forward projection: many independent problems in one persistent
 * launch.  The paper projects one volume at a time; a batch serves callers
 * with many small or uneven projections (several volumes, scan geometries,
 * storage types) whose separate launches would leave the GPU partly idle.
 */

/* One forward projection of a batch: the arguments of gjp_forward. */
typedef struct {
    const void *d_volume;         /* device [nx][ny][nz] elements of dtype */
    gjp_dtype dtype;
    int64_t nx, ny, nz;
    double voxel_size[3];         /* > 0 */
    double volume_origin[3];      /* world centre of voxel (0,0,0); used when has_origin != 0 */
    int has_origin;               /* 0: the centred grid */
    const gjp_geometry *geometry; /* its views, weight function and launch shape */
    float *d_proj;                /* device float32 [n_views][nv][nu], fully overwritten */
} gjp_problem;

/* Opaque, library-owned batch. */
typedef struct gjp_batch gjp_batch;

/*
 * gjp_batch_create -- validates `count` problems (1 .. 256; errors as for
 * gjp_forward, reported for the first bad problem) and prepares one work
 * queue over all of them: every problem is cut into items (one detector
 * tile of one view, 128 rays) and problems with the most planes per ray
 * are queued first.  Builds each geometry's device table on the current
 * device (as gjp_forward would) and allocates a few hundred bytes per
 * problem, plus a z-paired copy (4 bytes per voxel; see GJP_PATH_PAIRS and
 * gjp_batch_forward) for each bfloat16 or float16 problem that runs alone
 * where AUTO would take the copy -- a copy that cannot be allocated leaves its
 * problem reading the volume, with the same results.  The problems array
 * is copied, but the volumes, projections and geometries it points to must
 * stay valid while the batch is used.  Each
 * problem starts with its geometry's launch shape (gjp_geometry_set_launch;
 * a tile_u of 8 becomes 4).  Make this call before capturing a stream.
 */
gjp_status gjp_batch_create(const gjp_problem *problems, int count, gjp_batch **out);

/* Frees the batch (NULL-safe); waits for work that may still use it. */
void gjp_batch_destroy(gjp_batch *b);

/*
 * gjp_batch_forward -- the problems of the batch on `stream`: a problem
 * whose work items fill the GPU's resident blocks 16 times or more runs as
 * its own launch of the gather forward (the kernels of gjp_forward; a
 * bfloat16 or float16 one where AUTO would take the copy first rewrites its
 * z-paired copy, allocated by gjp_batch_create and kept with the batch), and all
 * other problems share one persistent kernel launch (preceded by a 4-byte
 * reset of the queue counter).  Nothing is allocated or synchronised, so
 * the call can be captured into a CUDA graph.  Each projection is bitwise
 * equal to
 * gjp_forward of the same problem (same per-ray arithmetic and warp
 * layout).  Batches share nothing, but two launches of the same batch must
 * not overlap on the GPU (they share the queue counter).  Returns
 * GJP_ERR_INVALID_ARG if the current device is not the one the batch was
 * created on.
 */
gjp_status gjp_batch_forward(const gjp_batch *b, void *stream);

/* The number of kernel launches one gjp_batch_forward makes (solo
 * problems' copy and gather launches, plus the persistent launch when the
 * queue holds problems; the counter reset is a memset, not a kernel). */
gjp_status gjp_batch_launch_count(const gjp_batch *b, int *launches);

/*
 * gjp_batch_autotune -- for every problem, times the batched launch of that
 * problem alone on its first 24 views for each tile shape (tile_u = 1, 2 or
 * 4 detector columns x 128/tile_u rows) and view interleaving (1, 4, 8, 16
 * views), `reps` timed runs after one warm-up each, and keeps the fastest.
 * Shapes that are fastest alone need not be fastest in the shared queue:
 * the whole batch is timed before and after, and the previous shapes are
 * restored if the tuned ones are slower.  A problem that runs as its own
 * launch takes the chosen tile_u as its blocks' detector columns (32 rows
 * each) and the chosen interleaving.  Writes valid projections and
 * synchronises `stream`; not for use during stream capture.  The choice
 * changes speed only, never a result.
 */
gjp_status gjp_batch_autotune(gjp_batch *b, void *stream, int reps);

/* Reads (get) or sets (set) the launch shape of problem `problem` (index
 * into the array given to gjp_batch_create).  tile_u: 1, 2 or 4;
 * view_group: 1 .. 64.  set uploads the new queue synchronously. */
gjp_status gjp_batch_get_tuning(const gjp_batch *b, int problem, int *tile_u, int *view_group);
gjp_status gjp_batch_set_tuning(gjp_batch *b, int problem, int tile_u, int view_group);

/* Static, human-readable name of a status code. */
const char *gjp_status_string(gjp_status s);

#ifdef __cplusplus
}
#endif

#endif /* GJP_H */
