// gjp_common.cuh -- declarations shared by the translation units of the
// GB300 GJP library: per-view and per-volume kernel parameters, launch
// constants, the geometry object, host helpers (defined in gjp.cu) and the
// per-ray device code of Algorithm 1 (setup, plane march, tap gather).
#pragma once

#include "gjp.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

namespace gjp_detail {

// ---------------------------------------------------------------------------
// Per-view device record: FP64 host quantities (index units; pixel
// coordinates centred on the panel, u = iu - (nu-1)/2, v = iv - (nv-1)/2)
// split into hi + lo FP32 parts.
struct ViewParams {
    float rh[9], rl[9];  // R0[3], RU[3], RV[3]: ray direction d - s (Eq. 2)
    float mh[9], ml[9];  // M0[3], MU[3], MV[3]: moment (s - c) x r about the centre c
};

struct VolParams {
    int n[3];
    float h[3];         // voxel size (world)
    long long s[3];     // element strides: ny*nz, nz, 1
    float fov_r2;       // > 0: squared world radius of the field-of-view cylinder (rays clipped to it)
};

#ifndef GJP_TILE_U
#define GJP_TILE_U 4
#endif
#ifndef GJP_BATCH
#define GJP_BATCH 4
#endif
#ifndef GJP_MIN_BLOCKS
#define GJP_MIN_BLOCKS 8      // 8 blocks of 128 threads: 64 registers per thread
#endif
#ifndef GJP_SLAB_MIN_BLOCKS
#define GJP_SLAB_MIN_BLOCKS 3
#endif
#ifndef GJP_ADJOINT_AUTO
#define GJP_ADJOINT_AUTO GJP_PATH_COMBINE   // adjoint family taken by GJP_PATH_AUTO
#endif
#ifndef GJP_VIEW_GROUP
#define GJP_VIEW_GROUP 16  // default launch order: 16 views per detector tile
#endif
// Warps whose 32 rays share their first transverse row step that row once
// per warp through a shared per-warp row table (1), or each lane steps its
// own copy (0); forward gather and warp-combined adjoint.
#ifndef GJP_ROWS
#define GJP_ROWS 1
#endif
// Debug build: GJP_CHECK_TAPS=1 range-checks every tap that the interior
// marches read or reduce without a per-tap test (their plane ranges come
// from the trimmed estimate of plane_interval).  A tap outside the grid is
// skipped and recorded in a device status word instead of being accessed;
// gjp_stream_status then reports GJP_ERR_INTERNAL.  Off by default: the
// production kernels carry no check.
#ifndef GJP_CHECK_TAPS
#define GJP_CHECK_TAPS 0
#endif
constexpr int kTileV = 32;          // lanes of a warp along v (contiguous z)
constexpr int kTileU = GJP_TILE_U;  // default warps of a block along u
#ifndef GJP_MAX_TILE_U
#define GJP_MAX_TILE_U 8
#endif
constexpr int kMaxTileU = GJP_MAX_TILE_U;   // largest block: 8 warps
constexpr int kMaxThreads = kTileV * kMaxTileU;
constexpr int kBatch = GJP_BATCH;   // interior planes per batch
static_assert(kBatch % 2 == 0, "interior batches are evaluated two planes at a time");
// the row-table march reads its 32-entry per-warp table in blocks of 4
// batches = 16 planes; other batch sizes would index past the table
static_assert(4 * kBatch == 16, "the row-table march is written for 4-plane batches");
// register budget of the one-thread-per-ray kernels: the same per-thread
// limit as GJP_MIN_BLOCKS resident blocks of 4 warps
constexpr int kMinBlocksMax = (GJP_MIN_BLOCKS * 4 + kMaxTileU - 1) / kMaxTileU;

struct gjp_cache_entry {
    int device;
    double key[9];
    ViewParams *d_table;
    int box_rows, box_cols4, box_cols8;   // slab box sizes for this grid (0 = not computed)
    void *tex = nullptr;                  // texture arrays of the texture families (gjp_texture.cu)
};

}  // namespace gjp_detail

struct gjp_geometry {
    int n_views, nu, nv;
    int weight = GJP_WEIGHT_LIN;          // interpolation weight function (Eq. 13 or Eq. 14)
    double fov = 0.0;                     // > 0: field-of-view cylinder radius (world units)
    int tile_u = gjp_detail::kTileU;                  // launch shape: warps (detector columns) per block
    int view_group = GJP_VIEW_GROUP;      // launch order: views interleaved per detector tile
    bool launch_set = false;              // set by the caller (else the view group follows the grid)
    double view_step = 0.0;               // median angle between consecutive views' central rays (radians)
    std::vector<double> src, org, du, dv;
    std::mutex mu;
    std::deque<gjp_detail::gjp_cache_entry> cache;   // deque: entries keep their address
};

namespace gjp_detail {

// ---------------------------------------------------------------------------
// Host helpers (gjp.cu).

// Host FP64 construction of the per-view table for one volume grid.
void build_table(const gjp_geometry &g, const int64_t n[3], const double h[3], const double o[3],
                 std::vector<ViewParams> &out);
// The device table for (g, current device, grid), built on first use.
gjp_status get_table(const gjp_geometry *g, const int64_t n[3], const double h[3], const double o[3],
                     gjp_cache_entry **out);
// Validates a volume grid; fills n, h and the origin (centred when origin is NULL).
gjp_status check_grid(int64_t nx, int64_t ny, int64_t nz, const double h[3], const double *origin,
                      int64_t n[3], double hh[3], double o[3]);
// Rejects a geometry with a source inside the interpolated support of the grid.
gjp_status check_sources(const gjp_geometry *g, const int64_t n[3], const double h[3], const double o[3]);
VolParams make_vol(const int64_t n[3], const double h[3], double fov);
// Whether every element offset the kernels form fits a signed 32-bit integer.
bool fits_int32(const int64_t n[3]);
// Sets func's preferred shared-memory carveout to the smallest share that
// still holds as many blocks of `threads` threads and `dyn_smem` dynamic
// bytes as its registers allow, leaving the rest of each SM's unified
// storage to the L1 cache.  (Left alone, the driver sizes the carveout for
// the thread-limited block count even where registers allow fewer blocks.)
// Once per function and device; a failure leaves the default in place.
void fit_carveout(const void *func, int threads, size_t dyn_smem);
size_t elem_size(gjp_dtype t);
// Launch shape of one gather forward launch (grid over the detector tiles
// of n_views views, view_group views interleaved per tile).
struct GatherShape {
    int nu, nv, n_views, tile_u, view_group;
    bool spl;
};
// The gather forward of one problem with an explicit launch shape (used by
// the batch for problems that fill the GPU alone): the row-table march reads
// its taps from `pairs` -- the problem's z-paired copy, already written by
// write_zpairs16; 16-bit storage, 32-bit offsets -- or from vol when null.
cudaError_t forward_gather_shaped(const void *vol, gjp_dtype dt, const VolParams &V, const ViewParams *table,
                                  const GatherShape &sh, bool i32, float *proj, const void *pairs, cudaStream_t s);
// Whether a 16-bit forward over n_views views of grid n is worth a z-paired
// copy (the rule AUTO follows; gjp.cu).
bool pairs_pay(int n_views, const int64_t n[3]);
// Writes the z-paired copy (4 bytes per voxel) of a bfloat16 or float16 volume.
cudaError_t write_zpairs16(const void *vol, gjp_dtype dt, const int64_t n[3], void *out, cudaStream_t s);
// Texture families (gjp_texture.cu): forward through the texture unit, and
// release of an entry's texture arrays (with the entry's device current).
gjp_status forward_texture(const void *d_volume, gjp_dtype dt, const int64_t n[3], const VolParams &V,
                           const gjp_geometry &g, gjp_cache_entry &entry, float *proj, int path, cudaStream_t s);
void free_texture_cache(gjp_cache_entry &e);
// Every device allocation of the library asks alloc_gate() first: false
// makes it fail as if the device were out of memory.  That happens only for
// the next n allocations after gjp_debug_fail_allocations(n), a test hook
// for the out-of-memory paths.
bool alloc_gate();
// An NVTX range around an entry point (no cost without a profiler attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
// Views interleaved per detector tile at launch: the caller's setting if it
// made one, else a default from the grid and the scan.  A view group's
// rays sweep nearly the same voxels, and its working set has to stay in the
// L2; it grows with the group's angular span and with the grid, so the span
// shrinks as the grid grows: 16 degrees at 512 voxels per edge, scaled by
// (512 / edge)^2, divided by the scan's step between views and held to
// 1 .. 16 views (measured on GB300 for the forward and the adjoint over 360
// views at 512, 640, 768, 896 and 1024 voxels per edge).
inline int launch_view_group(const gjp_geometry &g, const int n[3])
{
    if (g.launch_set) return g.view_group;
    const double m = (double)std::max(n[0], std::max(n[1], n[2]));
    const double span = 16.0 * (3.14159265358979323846 / 180.0) * (512.0 / m) * (512.0 / m);
    if (!(g.view_step > 1e-9)) return GJP_VIEW_GROUP;
    const double v = std::floor(span / g.view_step + 0.5);
    return (int)std::min<double>((double)GJP_VIEW_GROUP, std::max(1.0, v));
}
inline int launch_view_group(const gjp_geometry &g, const int64_t n[3])
{
    const int m[3] = {(int)std::min<int64_t>(n[0], INT_MAX), (int)std::min<int64_t>(n[1], INT_MAX),
                      (int)std::min<int64_t>(n[2], INT_MAX)};
    return launch_view_group(g, m);
}
// Tap-check faults recorded by the kernels of the other translation units
// (debug build; 0 otherwise), read and cleared.
unsigned batch_tap_faults();
unsigned texture_tap_faults();

// ---------------------------------------------------------------------------
// Device side: double-float helpers (error-free transformations with FMA).

struct f2 {
    float hi, lo;
};

__device__ __forceinline__ f2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ f2 quick_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ f2 f2_add(f2 x, f2 y)
{
    f2 s = two_sum(x.hi, y.hi);
    const f2 t = two_sum(x.lo, y.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ f2 f2_mul_f(f2 x, float f)
{
    const float p = __fmul_rn(x.hi, f);
    float e = __fmaf_rn(x.hi, f, -p);
    e = __fmaf_rn(x.lo, f, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ f2 f2_div(f2 x, f2 y)
{
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const f2 r = f2_add(x, f2_mul_f(y, -q1));
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return quick_two_sum(q1, q2);
}

__device__ __forceinline__ f2 f2_neg(f2 x) { return {-x.hi, -x.lo}; }

// X0[k] + u XU[k] + v XV[k] from a hi/lo coefficient block of 9 floats.
__device__ __forceinline__ f2 f2_affine(const float *h, const float *l, int k, float u, float v)
{
    const f2 x0 = {h[k], l[k]}, xu = {h[3 + k], l[3 + k]}, xv = {h[6 + k], l[6 + k]};
    return f2_add(f2_add(x0, f2_mul_f(xu, u)), f2_mul_f(xv, v));
}

// round(x * 2^32) as a 64-bit fixed-point number (|x| < 2^30).
__device__ __forceinline__ long long f2_to_fixed(f2 x)
{
    return __float2ll_rn(x.hi * 4294967296.0f) + __float2ll_rn(x.lo * 4294967296.0f);
}

template <typename X> __device__ __forceinline__ X sel3(X x0, X x1, X x2, int k)
{
    return k == 0 ? x0 : (k == 1 ? x1 : x2);
}

// Eq. 10: distance to the lower grid point, from the 32 fraction bits of a
// fixed-point position (top 23 bits placed in a float mantissa of [1, 2)).
__device__ __forceinline__ float frac_of(unsigned long long p)
{
    return __uint_as_float(__funnelshift_r((unsigned)p, 0x7Fu, 9)) - 1.0f;
}

__device__ __forceinline__ int floor_of(unsigned long long p) { return (int)(p >> 32); }

// Weight of the upper neighbour for distance d to the lower one: w_cl = 1 -
// w(d), which is d for w_lin (Eq. 13) and 3d^2 - 2d^3 for w_spl (Eq. 14).
template <bool SPL> __device__ __forceinline__ float upper_weight(float d)
{
    return SPL ? d * d * (3.0f - 2.0f * d) : d;
}

template <typename T> __device__ __forceinline__ float load_voxel(const T *p);
template <> __device__ __forceinline__ float load_voxel<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_voxel<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float load_voxel<__half>(const __half *p) { return __half2float(__ldg(p)); }

__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_float(__half x) { return __half2float(x); }

// ---------------------------------------------------------------------------
// Eq. 12 on packed FP32 pairs.  The interior marches evaluate two samples
// (planes t and t + 1 of a ray) per instruction with the paired FP32
// operations of sm_100+ (FFMA2), which halves the issue slots of the
// interpolation.  A 16-bit voxel stays in its storage word until the
// z-interpolation: the lower tap is widened (exact), and the difference to
// the upper tap is one mixed-precision subtraction (sub.f32.bf16 /
// sub.f32.f16: the 16-bit operand is widened exactly, one rounding), so
// weights and sums stay FP32 and the results equal those of widening every
// tap first.

template <typename T> struct Raw { using type = float; };
template <> struct Raw<__nv_bfloat16> { using type = unsigned short; };
template <> struct Raw<__half> { using type = unsigned short; };

template <typename T> __device__ __forceinline__ typename Raw<T>::type load_raw(const T *p)
{
    if constexpr (std::is_same<T, float>::value) return __ldg(p);
    else return __ldg(reinterpret_cast<const unsigned short *>(p));
}

template <typename T> __device__ __forceinline__ float widen(typename Raw<T>::type x)
{
    if constexpr (std::is_same<T, float>::value) return x;
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __uint_as_float((unsigned)x << 16);
    else return __half2float(__ushort_as_half(x));
}

// b - a, rounded once, for a stored voxel b and an FP32 a
template <typename T> __device__ __forceinline__ float sub_raw(typename Raw<T>::type b, float a)
{
    float r;
    if constexpr (std::is_same<T, float>::value) r = __fsub_rn(b, a);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(r) : "h"(b), "f"(a));
    else asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"(b), "f"(a));
    return r;
}

// Upper-neighbour weights (Eq. 10, 13/14) of two fixed-point positions.
template <bool SPL> __device__ __forceinline__ float2 upper_weight2(unsigned long long p, unsigned long long q)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 d = __fadd2_rn(make_float2(__uint_as_float(__funnelshift_r((unsigned)p, 0x7Fu, 9)),
                                            __uint_as_float(__funnelshift_r((unsigned)q, 0x7Fu, 9))),
                                m1);
    if (!SPL) return d;
    // 3d^2 - 2d^3 = d^2 (3 - 2d)
    return __fmul2_rn(__fmul2_rn(d, d), __ffma2_rn(d, make_float2(-2.0f, -2.0f), make_float2(3.0f, 3.0f)));
}

// Two samples of Eq. 12: taps (v00, v01) on the lower transverse row (lower
// and upper z), (v10, v11) on the upper row, for samples x and y of the
// pair; da / db the upper-neighbour weights of the row and z axes.
template <typename T>
__device__ __forceinline__ float2 eq12_pair(typename Raw<T>::type v00x, typename Raw<T>::type v00y,
                                            typename Raw<T>::type v01x, typename Raw<T>::type v01y,
                                            typename Raw<T>::type v10x, typename Raw<T>::type v10y,
                                            typename Raw<T>::type v11x, typename Raw<T>::type v11y, float2 da,
                                            float2 db)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 a0 = make_float2(widen<T>(v00x), widen<T>(v00y));
    const float2 a1 = make_float2(widen<T>(v10x), widen<T>(v10y));
    float2 d0, d1;
    if constexpr (std::is_same<T, float>::value) {
        d0 = __ffma2_rn(a0, m1, make_float2(v01x, v01y));   // v01 - v00
        d1 = __ffma2_rn(a1, m1, make_float2(v11x, v11y));
    } else {
        d0 = make_float2(sub_raw<T>(v01x, a0.x), sub_raw<T>(v01y, a0.y));
        d1 = make_float2(sub_raw<T>(v11x, a1.x), sub_raw<T>(v11y, a1.y));
    }
    const float2 e0 = __ffma2_rn(db, d0, a0);                 // lower row, interpolated along z
    const float2 e1 = __ffma2_rn(db, d1, a1);                 // upper row
    return __ffma2_rn(da, __ffma2_rn(e0, m1, e1), e0);      // between the rows
}

// ---------------------------------------------------------------------------
// The two z taps (z, z + 1) of one transverse row.  The row-table march
// reads them either from the volume itself (two loads) or from a z-paired
// copy of it, whose element e holds voxels e and e + 1 of the same z line
// (the upper one zero past the last z): one aligned 8-byte (float32) or
// 4-byte (16-bit) load then brings both taps, which halves the march's load
// instructions and, for 16-bit storage, its L1 wavefronts.  Both sources
// give the same tap values, so the results are bitwise equal.

template <typename T> struct PairOf { using type = float2; };
template <> struct PairOf<__nv_bfloat16> { using type = unsigned; };
template <> struct PairOf<__half> { using type = unsigned; };

template <typename T> struct ZTaps { typename Raw<T>::type lo, hi; };

#ifndef GJP_PAIRS_BATCH
#define GJP_PAIRS_BATCH 4
#endif
// planes per load batch of the row-table march: kBatch from the volume,
// GJP_PAIRS_BATCH from a z-paired copy (one word per row instead of two;
// 8-plane batches, which keep as many loads in flight as the volume's
// 4-plane ones, measured 0.8% slower for bfloat16 at 512^3)
template <typename S> constexpr int kRowBatch = kBatch;
template <> constexpr int kRowBatch<float2> = GJP_PAIRS_BATCH;
template <> constexpr int kRowBatch<unsigned> = GJP_PAIRS_BATCH;

template <typename T> __device__ __forceinline__ ZTaps<T> load_zrow(const T *p) { return {load_raw(p), load_raw(p + 1)}; }
__device__ __forceinline__ float2 load_zrow(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ unsigned load_zrow(const unsigned *p) { return __ldg(p); }

// the row's taps by source word: ZTaps<T> (plain), float2 or unsigned (paired)
template <typename T, typename Z> __device__ __forceinline__ void split_zrow(Z r, typename Raw<T>::type &lo,
                                                                             typename Raw<T>::type &hi)
{
    if constexpr (std::is_same<Z, ZTaps<T>>::value) {
        lo = r.lo;
        hi = r.hi;
    } else if constexpr (std::is_same<Z, float2>::value) {
        lo = r.x;
        hi = r.y;
    } else {
        asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(r));
    }
}

// Two samples of Eq. 12 from their rows' z-tap words: r0 (lower transverse
// row) and r1 (upper row) of samples x and y.
template <typename T, typename Z>
__device__ __forceinline__ float2 eq12_rows(Z r0x, Z r0y, Z r1x, Z r1y, float2 da, float2 db)
{
    typename Raw<T>::type v00x, v01x, v00y, v01y, v10x, v11x, v10y, v11y;
    split_zrow<T>(r0x, v00x, v01x);
    split_zrow<T>(r0y, v00y, v01y);
    split_zrow<T>(r1x, v10x, v11x);
    split_zrow<T>(r1y, v10y, v11y);
    return eq12_pair<T>(v00x, v00y, v01x, v01y, v10x, v10y, v11x, v11y, da, db);
}

// ---------------------------------------------------------------------------
// Per-ray setup.

struct Ray {
    int m, na, nb;            // driving axis (Eq. 3) and transverse extents
    int nm;                   // extent along m
    long long sm, sa, sb;     // element strides of m, a, b
    long long Pa, Pb;         // transverse positions at plane ic, fixed 32.32
    long long Ga, Gb;         // increments per plane (rt_a, rt_b of Eq. 4), fixed 32.32
    int ic;                   // anchor plane
    int s_lo, s_hi;           // planes with a possibly non-zero tap (support)
    int j_lo, j_hi;           // interior planes: all four taps inside the grid
    float step;               // |h (.) rt|: world length of one plane step
};

// ---------------------------------------------------------------------------
// Tap check of the debug build (GJP_CHECK_TAPS).  One status word per
// translation unit; take_tap_faults() reads and clears this unit's word.

static __device__ unsigned g_gjp_tap_fault;

// Whether the four taps of a sample with lower corner (ia, ib) on plane i lie
// in the grid (i in [0, nm), ia + 1 < na, ib + 1 < nb); records a violation.
// Always true, and free, in the production build.
__device__ __forceinline__ bool taps_in_grid(int i, int ia, int ib, int nm, int na, int nb)
{
    if (!GJP_CHECK_TAPS) return true;
    const bool ok = (unsigned)i < (unsigned)nm && ia >= 0 && ia + 1 < na && ib >= 0 && ib + 1 < nb;
    if (!ok) atomicOr(&g_gjp_tap_fault, 1u);
    return ok;
}

// The same for a row-table entry: `off` = i sm + ia sa (32-bit offsets) of
// plane i, z index ib.
__device__ __forceinline__ bool row_taps_in_grid(unsigned off, int i, int ib, const Ray &R)
{
    if (!GJP_CHECK_TAPS) return true;
    const unsigned rel = off - (unsigned)i * (unsigned)R.sm;
    const bool whole = rel % (unsigned)R.sa == 0u;
    const bool ok = whole && taps_in_grid(i, (int)(rel / (unsigned)R.sa), ib, R.nm, R.na, R.nb);
    if (!whole) atomicOr(&g_gjp_tap_fault, 1u);
    return ok;
}

static inline unsigned take_tap_faults()
{
#if GJP_CHECK_TAPS
    unsigned f = 0;
    if (cudaMemcpyFromSymbol(&f, g_gjp_tap_fault, sizeof f) != cudaSuccess) return 0;
    if (f) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(g_gjp_tap_fault, &z, sizeof z);
    }
    return f;
#else
    return 0;
#endif
}

__device__ __forceinline__ long long pos_at(long long P, long long G, int i, int ic)
{
    return P + (long long)(i - ic) * G;
}

// Planes i in [0, nm - 1] with lo < P + (i - ic) G < hi (fixed point,
// strict).  A float estimate brackets the crossings; the exact integer test
// then trims the bracket (positions are monotone in i).
__device__ __forceinline__ void plane_interval(long long P, long long G, int ic, long long lo, long long hi,
                                               int nm, int &a, int &b)
{
    if (G == 0) {
        const bool in = lo < P && P < hi;
        a = 0;
        b = in ? nm - 1 : -1;
        return;
    }
    const float g = __ll2float_rn(G);
    const float t1 = __ll2float_rn(lo - P) / g, t2 = __ll2float_rn(hi - P) / g;
    const float lim = 3.0e7f;
    const float tmin = fmaxf(fminf(t1, t2), -lim), tmax = fminf(fmaxf(t1, t2), lim);
    a = max(0, ic + (int)floorf(tmin) - 2);
    b = min(nm - 1, ic + (int)ceilf(tmax) + 2);
    while (a <= b) {
        const long long p = pos_at(P, G, a, ic);
        if (lo < p && p < hi) break;
        ++a;
    }
    while (b >= a) {
        const long long p = pos_at(P, G, b, ic);
        if (lo < p && p < hi) break;
        --b;
    }
}

// Field-of-view cylinder (the speed section samples each ray only on its
// intersection with a cylinder around the rotation axis): keeps the planes
// whose sample lies within world radius sqrt(fov_r2) of the axis through
// the volume centre parallel to z.  The sample's (x, y) is affine in the
// plane index t = i - ic, so the kept planes are the integers between the
// two roots of a quadratic (float32; a sample within ~1e-4 plane of the
// circle may fall on either side, which cannot matter for a volume that is
// zero near the cylinder wall, the setting this option is for).
__device__ __forceinline__ void clip_to_fov(const VolParams &V, Ray &R, int m)
{
    const float inv = 2.3283064365386963e-10f;   // 2^-32
    // index position at t = 0 and per plane, for x and y
    float p0[2], dp[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool is_m = k == m, is_a = k == ((m == 0) ? 1 : 0);
        p0[k] = is_m ? (float)R.ic : __ll2float_rn(is_a ? R.Pa : R.Pb) * inv;
        dp[k] = is_m ? 1.0f : __ll2float_rn(is_a ? R.Ga : R.Gb) * inv;
    }
    const float X0 = V.h[0] * (p0[0] - 0.5f * (float)(V.n[0] - 1)), dX = V.h[0] * dp[0];
    const float Y0 = V.h[1] * (p0[1] - 0.5f * (float)(V.n[1] - 1)), dY = V.h[1] * dp[1];
    const float A = dX * dX + dY * dY, B = X0 * dX + Y0 * dY, C = X0 * X0 + Y0 * Y0 - V.fov_r2;
    int lo, hi;
    if (A <= 0.0f) {                       // no motion in (x, y): all planes or none
        lo = C <= 0.0f ? 0 : 1;
        hi = C <= 0.0f ? 0x3fffffff : 0;
    } else {
        const float disc = B * B - A * C;
        if (disc < 0.0f) {
            lo = 1;
            hi = 0;
        } else {
            const float sq = sqrtf(disc);
            const float t1 = (-B - sq) / A, t2 = (-B + sq) / A;
            lo = R.ic + (int)ceilf(fmaxf(t1, -1.0e9f));
            hi = R.ic + (int)floorf(fminf(t2, 1.0e9f));
        }
    }
    R.s_lo = max(R.s_lo, lo);
    R.s_hi = min(R.s_hi, hi);
    R.j_lo = max(R.j_lo, lo);
    R.j_hi = min(R.j_hi, hi);
}

__device__ __forceinline__ void setup_ray(const ViewParams &vp, const VolParams &V, float u, float v, Ray &R)
{
    const f2 r0 = f2_affine(vp.rh, vp.rl, 0, u, v);
    const f2 r1 = f2_affine(vp.rh, vp.rl, 1, u, v);
    const f2 r2 = f2_affine(vp.rh, vp.rl, 2, u, v);
    int m = 0;                                           // Eq. 3, ties to the lowest index
    if (fabsf(r1.hi) > fabsf(r0.hi)) m = 1;
    if (fabsf(r2.hi) > fabsf(sel3(r0.hi, r1.hi, r2.hi, m))) m = 2;
    const int a = (m == 0) ? 1 : 0;
    const int b = (m == 2) ? 1 : 2;
    const f2 rm = sel3(r0, r1, r2, m), ra = sel3(r0, r1, r2, a), rb = sel3(r0, r1, r2, b);
    // moment components L_a, L_b: the centre-plane crossing is
    // q_a = -+ L_b / r_m, q_b = -+ L_a / r_m  (minus for the cyclic order (m, k, j))
    const f2 L0 = f2_affine(vp.mh, vp.ml, 0, u, v);
    const f2 L1 = f2_affine(vp.mh, vp.ml, 1, u, v);
    const f2 L2 = f2_affine(vp.mh, vp.ml, 2, u, v);
    const f2 La = sel3(L0, L1, L2, a), Lb = sel3(L0, L1, L2, b);
    f2 qa = f2_div(Lb, rm), qb = f2_div(La, rm);
    if (a == (m + 1) % 3) qa = f2_neg(qa);
    if (b == (m + 1) % 3) qb = f2_neg(qb);
    const f2 ga = f2_div(ra, rm), gb = f2_div(rb, rm);   // Eq. 4

    const int nm = sel3(V.n[0], V.n[1], V.n[2], m);
    R.m = m;
    R.nm = nm;
    R.na = sel3(V.n[0], V.n[1], V.n[2], a);
    R.nb = sel3(V.n[0], V.n[1], V.n[2], b);
    R.sm = sel3(V.s[0], V.s[1], V.s[2], m);
    R.sa = sel3(V.s[0], V.s[1], V.s[2], a);
    R.sb = sel3(V.s[0], V.s[1], V.s[2], b);
    const float cm = 0.5f * (float)(nm - 1);
    R.ic = (nm - 1) >> 1;                                 // floor(c_m)
    const float delta = (float)R.ic - cm;                 // 0 or -1/2
    const f2 Pa = f2_add(f2_add(qa, {0.5f * (float)(R.na - 1), 0.0f}), f2_mul_f(ga, delta));
    const f2 Pb = f2_add(f2_add(qb, {0.5f * (float)(R.nb - 1), 0.0f}), f2_mul_f(gb, delta));
    R.Pa = f2_to_fixed(Pa);
    R.Pb = f2_to_fixed(Pb);
    R.Ga = f2_to_fixed(ga);
    R.Gb = f2_to_fixed(gb);
    const float hm = sel3(V.h[0], V.h[1], V.h[2], m);
    const float ha = sel3(V.h[0], V.h[1], V.h[2], a) * ga.hi, hb = sel3(V.h[0], V.h[1], V.h[2], b) * gb.hi;
    R.step = sqrtf(hm * hm + ha * ha + hb * hb);

    // support: -1 < p < n on both transverse axes; interior: 0 <= p < n - 1
    const long long one = 1LL << 32;
    int sa0, sa1, sb0, sb1, ja0, ja1, jb0, jb1;
    plane_interval(R.Pa, R.Ga, R.ic, -one, (long long)R.na * one, nm, sa0, sa1);
    plane_interval(R.Pb, R.Gb, R.ic, -one, (long long)R.nb * one, nm, sb0, sb1);
    plane_interval(R.Pa, R.Ga, R.ic, -1, (long long)(R.na - 1) * one, nm, ja0, ja1);
    plane_interval(R.Pb, R.Gb, R.ic, -1, (long long)(R.nb - 1) * one, nm, jb0, jb1);
    R.s_lo = max(sa0, sb0);
    R.s_hi = min(sa1, sb1);
    R.j_lo = max(max(ja0, jb0), R.s_lo);
    R.j_hi = min(min(ja1, jb1), R.s_hi);
    if (V.fov_r2 > 0.0f) clip_to_fov(V, R, m);
}

__device__ __forceinline__ void load_view(const ViewParams *__restrict__ views, int k, ViewParams &vp)
{
    const float *src = reinterpret_cast<const float *>(views + k);
    float *dst = reinterpret_cast<float *>(&vp);
#pragma unroll
    for (int j = 0; j < 36; ++j) dst[j] = __ldg(src + j);
}

// Boundary planes: the support planes outside the interior range, visited
// as one index list (before the interior, then after it).
__device__ __forceinline__ int boundary_count(const Ray &R, int &n_before)
{
    if (R.s_lo > R.s_hi) {
        n_before = 0;
        return 0;
    }
    if (R.j_lo > R.j_hi) {
        n_before = R.s_hi - R.s_lo + 1;
        return n_before;
    }
    n_before = R.j_lo - R.s_lo;
    return n_before + (R.s_hi - R.j_hi);
}

__device__ __forceinline__ int boundary_plane(const Ray &R, int k, int n_before)
{
    return k < n_before ? R.s_lo + k : R.j_hi + 1 + (k - n_before);
}

// ---------------------------------------------------------------------------
// Block order.  The grid is (detector tiles, views); blocks are numbered
// linearly (x fastest) and dispatched roughly in that order.  With
// view_group = G the linear number is mapped so that G consecutive blocks
// cover the same detector tile of G consecutive views: rays of neighbouring
// views through the same tile sweep nearly the same voxels at nearly the
// same time, so the L2 cache serves the later views' taps.  G = 1 is plain
// view-major order.
__device__ __forceinline__ void block_tile_view(int n_views, int view_group, int &tile, int &view)
{
    const long long n_tiles = gridDim.x;
    const long long L = (long long)blockIdx.y * n_tiles + blockIdx.x;
    const long long per = n_tiles * view_group;
    const int grp = (int)(L / per);
    const int r = (int)(L - (long long)grp * per);
    const int v0 = grp * view_group;
    const int gl = min(view_group, n_views - v0);   // last group may hold fewer views
    view = v0 + r % gl;
    tile = r / gl;
}

// ---------------------------------------------------------------------------
// Forward projection: one thread per ray; a block is blockDim.y detector
// columns x 32 rows (v-tiles fastest within a view).

// One batch of kBatch interior planes of a ray (no checks): gathers the
// 4 kBatch taps first, then evaluates Eq. 12 two planes at a time; returns
// the batch sum as an FP32 pair (even and odd planes).
template <typename T, typename Index, bool SPL>
__device__ __forceinline__ float2 interior_batch(const T *__restrict__ vol, unsigned long long &pa,
                                                 unsigned long long &pb, Index &plane, unsigned long long ga,
                                                 unsigned long long gb, Index sa, Index sb, Index sm, int &ii,
                                                 int di, const Ray &R)
{
    using W = typename Raw<T>::type;
    W v00[kBatch], v01[kBatch], v10[kBatch], v11[kBatch];
    unsigned long long qa[kBatch], qb[kBatch];
#pragma unroll
    for (int t = 0; t < kBatch; ++t) {
        qa[t] = pa;
        qb[t] = pb;
        const bool ok = taps_in_grid(ii, floor_of(pa), floor_of(pb), R.nm, R.na, R.nb);   // debug build only
        const T *p = vol + (plane + (Index)floor_of(pa) * sa + (Index)floor_of(pb) * sb);
        v00[t] = ok ? load_raw(p) : W(0);
        v01[t] = ok ? load_raw(p + sb) : W(0);
        v10[t] = ok ? load_raw(p + sa) : W(0);
        v11[t] = ok ? load_raw(p + sa + sb) : W(0);
        pa += ga;
        pb += gb;
        plane += sm;
        ii += di;
    }
    float2 bsum = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int t = 0; t < kBatch; t += 2) {
        const float2 da = upper_weight2<SPL>(qa[t], qa[t + 1]), db = upper_weight2<SPL>(qb[t], qb[t + 1]);
        bsum = __fadd2_rn(bsum, eq12_pair<T>(v00[t], v00[t + 1], v01[t], v01[t + 1], v10[t], v10[t + 1], v11[t],
                                             v11[t + 1], da, db));
    }
    return bsum;
}

// Interior planes j_lo .. j_hi of one ray: all four taps lie inside the
// grid, so no checks.  rev marches the same planes from j_hi down to j_lo
// (a warp picks the direction in which its lanes start on a common plane,
// so that they read neighbouring voxels together).
template <typename T, typename Index, bool ZB, bool SPL = false>
__device__ __forceinline__ float march_interior(const T *__restrict__ vol, const Ray &R, bool rev = false)
{
    // ZB: the second transverse axis is z (stride 1), true unless m == z
    const Index sa = (Index)R.sa;
    const Index sb = ZB ? (Index)1 : (Index)R.sb;
    const int i0 = rev ? R.j_hi : R.j_lo;
    int count = R.j_hi - R.j_lo + 1;
    unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, i0, R.ic);
    unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, i0, R.ic);
    const unsigned long long ga = rev ? 0ull - (unsigned long long)R.Ga : (unsigned long long)R.Ga;
    const unsigned long long gb = rev ? 0ull - (unsigned long long)R.Gb : (unsigned long long)R.Gb;
    const Index sm = rev ? -(Index)R.sm : (Index)R.sm;
    Index plane = (Index)i0 * (Index)R.sm;
    int ii = i0;                                     // plane index (checked in the debug build)
    const int di = rev ? -1 : 1;
    // two-level sum: planes of a batch are added together, four batch sums
    // make a block sum, and block sums join the total once per 16 planes
    // (float32 error ~4x smaller than a running sum over up to ~n_m planes);
    // the partial sums are FP32 pairs (even and odd planes)
    float2 acc = make_float2(0.0f, 0.0f);
    for (; count >= 4 * kBatch; count -= 4 * kBatch) {
        float2 blk = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            blk = __fadd2_rn(blk, interior_batch<T, Index, SPL>(vol, pa, pb, plane, ga, gb, sa, sb, sm, ii, di, R));
        acc = __fadd2_rn(acc, blk);
    }
    float2 part = make_float2(0.0f, 0.0f);           // fewer than 16 planes left
    for (; count >= kBatch; count -= kBatch)
        part = __fadd2_rn(part, interior_batch<T, Index, SPL>(vol, pa, pb, plane, ga, gb, sa, sb, sm, ii, di, R));
    acc = __fadd2_rn(acc, part);
    float tail = 0.0f;
    for (; count > 0; --count) {
        const float da = upper_weight<SPL>(frac_of(pa)), db = upper_weight<SPL>(frac_of(pb));
        const bool ok = taps_in_grid(ii, floor_of(pa), floor_of(pb), R.nm, R.na, R.nb);
        const T *p = vol + (plane + (Index)floor_of(pa) * sa + (Index)floor_of(pb) * sb);
        const float v00 = ok ? load_voxel(p) : 0.0f, v01 = ok ? load_voxel(p + sb) : 0.0f;
        const float v10 = ok ? load_voxel(p + sa) : 0.0f, v11 = ok ? load_voxel(p + sa + sb) : 0.0f;
        const float e0 = __fmaf_rn(db, v01 - v00, v00);
        const float e1 = __fmaf_rn(db, v11 - v10, v10);
        tail += __fmaf_rn(da, e1 - e0, e0);
        pa += ga;
        pb += gb;
        plane += sm;
        ii += di;
    }
    return (acc.x + acc.y) + tail;
}

template <typename T, typename Index, bool SPL = false>
__device__ __forceinline__ float march_boundary(const T *__restrict__ vol, const Ray &R)
{
    int n_before;
    const int nbd = boundary_count(R, n_before);
    const Index sa = (Index)R.sa, sb = (Index)R.sb, sm = (Index)R.sm;
    const unsigned na = (unsigned)R.na, nb = (unsigned)R.nb;
    float acc = 0.0f;
    for (int k = 0; k < nbd; ++k) {
        const int i = boundary_plane(R, k, n_before);
        const unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, i, R.ic);
        const unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, i, R.ic);
        const float da = upper_weight<SPL>(frac_of(pa)), db = upper_weight<SPL>(frac_of(pb));
        const int ia = floor_of(pa), ib = floor_of(pb);
        const bool a0 = (unsigned)ia < na, a1 = (unsigned)(ia + 1) < na;   // zero border
        const bool b0 = (unsigned)ib < nb, b1 = (unsigned)(ib + 1) < nb;
        const T *p = vol + ((Index)i * sm + (Index)ia * sa + (Index)ib * sb);
        const float v00 = (a0 && b0) ? load_voxel(p) : 0.0f;
        const float v01 = (a0 && b1) ? load_voxel(p + sb) : 0.0f;
        const float v10 = (a1 && b0) ? load_voxel(p + sa) : 0.0f;
        const float v11 = (a1 && b1) ? load_voxel(p + sa + sb) : 0.0f;
        const float e0 = __fmaf_rn(db, v01 - v00, v00);
        const float e1 = __fmaf_rn(db, v11 - v10, v10);
        acc += __fmaf_rn(da, e1 - e0, e0);
    }
    return acc;
}

// One 16-plane block of the row-table march (below): e holds, per pair of
// planes (t, t + 1), the words (row weight t, row weight t + 1, row offset
// t, row offset t + 1), read with one 16-byte load; pb steps along z.  src
// is the volume (S = T) or its z-paired copy (S = PairOf<T>::type), indexed
// alike.  CHECKED loads only the taps of planes 0 <= d + t < cnt (this
// lane's interior), the others contribute zero, and stops after `n` planes
// (warp-uniform: no lane has an interior plane past them).  Returns the
// block sum as an FP32 pair (even and odd planes).
template <typename T, bool SPL, bool CHECKED, int B, typename S>
__device__ __forceinline__ float2 rows_block(const S *__restrict__ src, const uint4 *__restrict__ e,
                                             unsigned long long &pb, unsigned long long gb, int sa, int d, int cnt,
                                             int n, int ip, int dir, const Ray &R)
{
    // (ip, dir: plane index of entry 0 and the march direction, for the
    // tap check of the debug build; B: planes whose taps are loaded before
    // their arithmetic, 16 / B such batches)
    static_assert(B % 2 == 0 && 16 % B == 0, "load batches split the 16-plane block");
    using Z = decltype(load_zrow(src));
    float2 blk = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < 16 / B; ++q) {
        if (CHECKED && q * B >= n) break;
        Z r0[B], r1[B];                              // lower / upper transverse row
        unsigned long long qb[B];
        float2 da[B / 2];
        unsigned off[B];
#pragma unroll
        for (int t = 0; t < B; t += 2) {
            const uint4 en = e[(q * B + t) / 2];
            da[t / 2] = make_float2(__uint_as_float(en.x), __uint_as_float(en.y));
            off[t] = en.z;
            off[t + 1] = en.w;
        }
#pragma unroll
        for (int t = 0; t < B; ++t) {
            qb[t] = pb;
            const S *p = src + (int)(off[t] + (unsigned)floor_of(pb));
            const int i = ip + dir * (q * B + t);
            const bool in = CHECKED ? (unsigned)(d + q * B + t) < (unsigned)cnt &&
                                          (!GJP_CHECK_TAPS || row_taps_in_grid(off[t], i, floor_of(pb), R))
                                    : row_taps_in_grid(off[t], i, floor_of(pb), R);   // debug build only
            r0[t] = in ? load_zrow(p) : Z{};
            r1[t] = in ? load_zrow(p + sa) : Z{};
            pb += gb;
        }
#pragma unroll
        for (int t = 0; t < B; t += 2) {
            const float2 db = upper_weight2<SPL>(qb[t], qb[t + 1]);
            blk = __fadd2_rn(blk, eq12_rows<T>(r0[t], r0[t + 1], r1[t], r1[t + 1], da[t / 2], db));
        }
    }
    return blk;
}

// Interior planes of a warp whose 32 rays share their first transverse row:
// the same driving axis (x or y, so the second transverse axis is z), the
// same Pa and the same Ga -- every ray of a detector column when the orbit
// turns about z.  The row index ia, its weight and the plane's offset are
// then the same on every lane, so the warp computes each plane's row once:
// lane k fills the entry of the k-th of the next 32 planes, and every lane
// reads the entries with broadcast shared-memory loads instead of stepping,
// splitting and scaling its own copy of the row position.  The lanes march
// the warp's planes together; a 16-plane block inside every lane's interior
// runs without checks, other blocks load only the taps of lanes whose
// interior holds the plane (their boundary planes are summed elsewhere).
// `rows` is this warp's 32-entry table (256 bytes, 16-byte aligned): per
// pair of planes the row weight bits of both, then the row offsets of both
// (the layout rows_block reads).
template <typename T, bool SPL, typename S>
__device__ __forceinline__ float march_interior_rows(const S *__restrict__ src, const Ray &R, bool rev,
                                                     uint4 *__restrict__ rows, int lane)
{
    const unsigned full = 0xffffffffu;
    const bool has = R.j_lo <= R.j_hi;
    const int I0 = __reduce_min_sync(full, has ? R.j_lo : INT_MAX);
    const int I1 = __reduce_max_sync(full, has ? R.j_hi : INT_MIN);
    if (I0 > I1) return 0.0f;                         // no lane has an interior plane (warp-uniform)
    const int L = I1 - I0 + 1;                        // step k visits plane i0 + dir k
    const int i0 = rev ? I1 : I0, dir = rev ? -1 : 1;
    const int cnt = has ? R.j_hi - R.j_lo + 1 : 0;   // this lane: steps k_lo .. k_lo + cnt - 1
    const int k_lo = rev ? I1 - R.j_hi : R.j_lo - I0;
    // steps at which every lane is interior (none when a lane has no interior)
    const int K0 = __reduce_max_sync(full, has ? k_lo : INT_MAX);
    const int K1 = __reduce_min_sync(full, has ? k_lo + cnt - 1 : INT_MIN);

    const int sa = R.sa;
    unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, i0, R.ic);
    const unsigned long long gb = rev ? 0ull - (unsigned long long)R.Gb : (unsigned long long)R.Gb;
    // this lane's table plane in window w: i0 + dir (32 w + lane); offsets in
    // unsigned arithmetic (planes past the warp's range are filled, never read)
    unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, i0 + dir * lane, R.ic);
    const unsigned long long ga32 = (rev ? 0ull - (unsigned long long)R.Ga : (unsigned long long)R.Ga) << 5;
    unsigned row = (unsigned)(i0 + dir * lane) * (unsigned)R.sm;
    const unsigned sm32 = (unsigned)(dir * 32) * (unsigned)R.sm;

    unsigned *slot = reinterpret_cast<unsigned *>(rows) + 4 * (lane >> 1) + (lane & 1);
    float2 acc = make_float2(0.0f, 0.0f);
    for (int w = 0; w < L; w += 32) {
        __syncwarp();                                 // every lane has read the last window
        slot[0] = __float_as_uint(upper_weight<SPL>(frac_of(pa)));
        slot[2] = row + (unsigned)floor_of(pa) * (unsigned)sa;
        pa += ga32;
        row += sm32;
        __syncwarp();
        const int nw = min(32, L - w);
        for (int kb = 0; kb < nw; kb += 16) {
            const int k = w + kb;
            const int ip = i0 + dir * k;
            if (k >= K0 && k + 15 <= K1)              // warp-uniform
                acc = __fadd2_rn(acc, rows_block<T, SPL, false, kRowBatch<S>>(src, rows + kb / 2, pb, gb, sa, 0, 0, 16,
                                                                             ip, dir, R));
            else
                acc = __fadd2_rn(acc, rows_block<T, SPL, true, kRowBatch<S>>(src, rows + kb / 2, pb, gb, sa, k - k_lo, cnt, L - k,
                                                               ip, dir, R));
        }
    }
    return acc.x + acc.y;
}

// Row tables of the row-table march: 32 entries of 8 bytes per warp slot at
// the start of the dynamic shared memory.  Reached through this symbol (not
// a pointer handed down) so that every table access compiles to a
// shared-memory access.
extern __shared__ uint4 gjp_row_tables[];

__device__ __forceinline__ uint2 *row_table(int slot) { return reinterpret_cast<uint2 *>(gjp_row_tables + 16 * slot); }

__device__ __forceinline__ int lane_id()
{
    int l;
    asm("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}

// GJP line integral of the ray through detector pixel (iu, iv) of the view
// whose table entry is *view (Algorithm 1).  Called by every lane of the
// warp set in `act` (the lanes that hold a ray; they share the warp-level
// choice of march direction).  PAIRS: the row-table march reads its taps
// from `pairs`, the z-paired copy of vol (32-bit offsets only).
template <typename T, typename Index, bool SPL, bool PAIRS = false>
__device__ __forceinline__ float forward_ray(const T *__restrict__ vol, const VolParams &V,
                                             const ViewParams *__restrict__ view, int nu, int nv, int iu, int iv,
                                             unsigned act, int rows_slot = -1,
                                             const typename PairOf<T>::type *__restrict__ pairs = nullptr)
{
    ViewParams vp;
    load_view(view, 0, vp);
    Ray R;
    setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);

    // March direction: the lanes of a warp usually enter their interior
    // planes together at one end and leave at different planes at the other
    // (rays of a detector column cross the top or bottom face of the volume
    // one after another).  Starting at the end where the lanes agree keeps
    // them on a common plane, so their taps fall on neighbouring voxels.
    const int lo_spread = __reduce_max_sync(act, R.j_lo) - __reduce_min_sync(act, R.j_lo);
    const int hi_spread = __reduce_max_sync(act, R.j_hi) - __reduce_min_sync(act, R.j_hi);
    const bool rev = hi_spread < lo_spread;

    // the few boundary planes first: afterwards only the interior march's
    // state stays live, which keeps the unrolled loop within the register budget
    const float bsum = march_boundary<T, Index, SPL>(vol, R);
    static_assert(!PAIRS || std::is_same<Index, int>::value, "the z-paired copy is read with 32-bit offsets");
    if constexpr (std::is_same<Index, int>::value) {
        // a full warp with one common row: the shared row table
        if (GJP_ROWS && rows_slot >= 0 && act == 0xffffffffu) {
            const int m0 = __shfl_sync(act, R.m, 0);
            const long long Pa0 = __shfl_sync(act, R.Pa, 0), Ga0 = __shfl_sync(act, R.Ga, 0);
            if (__all_sync(act, R.m == m0 && R.Pa == Pa0 && R.Ga == Ga0) && m0 != 2) {
                uint4 *rows = gjp_row_tables + 16 * rows_slot;
                const float acc = PAIRS ? march_interior_rows<T, SPL>(pairs, R, rev, rows, lane_id())
                                        : march_interior_rows<T, SPL>(vol, R, rev, rows, lane_id());
                return (acc + bsum) * R.step;
            }
        }
    }
    const float acc = (R.m != 2) ? march_interior<T, Index, true, SPL>(vol, R, rev)
                                 : march_interior<T, Index, false, SPL>(vol, R, rev);
    return (acc + bsum) * R.step;
}

}  // namespace gjp_detail
