// gjp.cu -- GB300 (sm_103a) branchless generalized Joseph projector:
// host-side geometry (FP64), forward / adjoint / footprint kernels, and the
// C ABI declared in include/gjp.h.
//
// Method: Algorithm 1 (Eq. 1-13) of Graetz, "High performance volume ray
// casting: A branchless generalized Joseph projector".  Each thread owns one
// ray (one detector pixel of one view), marches the integer planes
// perpendicular to its driving axis m and accumulates the bilinearly
// interpolated volume, scaled by the world length of one plane step.
//
// GB300 design points:
//  * Per-view constants are formed in FP64 on the host and shipped as
//    hi/lo FP32 pairs: the ray direction r(u, v) = R0 + u RU + v RV and the
//    moment of the ray about the volume centre, L(u, v) = (s - c) x r.  The
//    crossing of the centre plane follows from L / r_m, which avoids the
//    cancellation of s + (o + i) rt when |s| is several volume widths.
//  * The per-ray setup runs in double-float arithmetic (pairs of FP32, on
//    the FP32 pipes; GB300's FP64 rate is very low) and leaves the two
//    transverse positions and their per-plane increments as 64-bit fixed
//    point numbers with 32 fraction bits.  Stepping is an exact integer add;
//    the integer part is the floor of Eq. 7 and the fraction is Eq. 10's
//    distance, so sample positions carry ~1e-7 voxel error at any volume
//    size, with no float-to-int conversions in the loop.
//  * The driving-axis coordinate of every sample is the plane index itself
//    (an exact integer, as Algorithm 1 asserts).
//  * Each ray's plane range is split exactly (integer arithmetic) into the
//    interior planes, where all four taps lie in the grid and no bounds
//    checks are needed, and the few boundary planes, where taps outside the
//    grid read zero.  Interior planes are processed four at a time so each
//    thread keeps 16 independent loads in flight.
//  * Warps run along detector v, which maps to the contiguous z index of the
//    volume: lanes of a warp read consecutive voxels (the memory-order rule
//    that accompanies Algorithm 1).
#include "gjp.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

namespace {

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
};

#ifndef GJP_TILE_U
#define GJP_TILE_U 8
#endif
#ifndef GJP_BATCH
#define GJP_BATCH 4
#endif
constexpr int kTileV = 32;          // lanes of a warp along v (contiguous z)
constexpr int kTileU = GJP_TILE_U;  // warps of a block along u
constexpr int kThreads = kTileV * kTileU;
constexpr int kBatch = GJP_BATCH;   // interior planes per batch

struct gjp_cache_entry {
    int device;
    double key[9];
    ViewParams *d_table;
};

}  // namespace

struct gjp_geometry {
    int n_views, nu, nv;
    std::vector<double> src, org, du, dv;
    std::mutex mu;
    std::vector<gjp_cache_entry> cache;
};

namespace {

bool finite3(const double *p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

void split(double x, float &hi, float &lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// Host FP64 construction of the per-view table for one volume grid.
void build_table(const gjp_geometry &g, const int64_t n[3], const double h[3], const double o[3],
                 std::vector<ViewParams> &out)
{
    out.resize(g.n_views);
    const double cu = 0.5 * (g.nu - 1), cv = 0.5 * (g.nv - 1);
    for (int k = 0; k < g.n_views; ++k) {
        double s[3], R[9], M[9];
        for (int a = 0; a < 3; ++a) {
            const double c = 0.5 * (double)(n[a] - 1);
            s[a] = (g.src[3 * k + a] - o[a]) / h[a] - c;                     // source, centred index units
            R[3 + a] = g.du[3 * k + a] / h[a];
            R[6 + a] = g.dv[3 * k + a] / h[a];
            R[a] = (g.org[3 * k + a] - g.src[3 * k + a]) / h[a] + cu * R[3 + a] + cv * R[6 + a];
        }
        for (int t = 0; t < 3; ++t) {                                         // M = s x R (columns 0,1,2)
            const double *x = R + 3 * t;
            M[3 * t + 0] = s[1] * x[2] - s[2] * x[1];
            M[3 * t + 1] = s[2] * x[0] - s[0] * x[2];
            M[3 * t + 2] = s[0] * x[1] - s[1] * x[0];
        }
        ViewParams &vp = out[k];
        for (int j = 0; j < 9; ++j) {
            split(R[j], vp.rh[j], vp.rl[j]);
            split(M[j], vp.mh[j], vp.ml[j]);
        }
    }
}

// Returns the device table for (g, current device, grid); builds it on first use.
gjp_status get_table(const gjp_geometry *gc, const int64_t n[3], const double h[3], const double o[3],
                     const ViewParams **out)
{
    gjp_geometry *g = const_cast<gjp_geometry *>(gc);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GJP_ERR_CUDA;
    double key[9] = {(double)n[0], (double)n[1], (double)n[2], h[0], h[1], h[2], o[0], o[1], o[2]};
    std::lock_guard<std::mutex> lock(g->mu);
    for (const auto &e : g->cache) {
        if (e.device == dev && std::memcmp(e.key, key, sizeof key) == 0) {
            *out = e.d_table;
            return GJP_OK;
        }
    }
    std::vector<ViewParams> host;
    try {
        build_table(*g, n, h, o, host);
    } catch (const std::bad_alloc &) {
        return GJP_ERR_OOM;
    }
    ViewParams *d = nullptr;
    const size_t bytes = sizeof(ViewParams) * host.size();
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        return GJP_ERR_OOM;
    }
    if (cudaMemcpy(d, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return GJP_ERR_CUDA;
    }
    gjp_cache_entry e;
    e.device = dev;
    std::memcpy(e.key, key, sizeof key);
    e.d_table = d;
    g->cache.push_back(e);
    *out = d;
    return GJP_OK;
}

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

template <typename T> __device__ __forceinline__ float load_voxel(const T *p);
template <> __device__ __forceinline__ float load_voxel<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_voxel<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float load_voxel<__half>(const __half *p) { return __half2float(__ldg(p)); }

// ---------------------------------------------------------------------------
// Per-ray setup.

struct Ray {
    int m, na, nb;            // driving axis (Eq. 3) and transverse extents
    long long sm, sa, sb;     // element strides of m, a, b
    long long Pa, Pb;         // transverse positions at plane ic, fixed 32.32
    long long Ga, Gb;         // increments per plane (rt_a, rt_b of Eq. 4), fixed 32.32
    int ic;                   // anchor plane
    int s_lo, s_hi;           // planes with a possibly non-zero tap (support)
    int j_lo, j_hi;           // interior planes: all four taps inside the grid
    float step;               // |h (.) rt|: world length of one plane step
};

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
// Forward projection: one thread per ray; blockIdx.x = detector tile
// (v-tiles fastest), blockIdx.y = view.

template <typename T, typename Index, bool ZB>
__device__ __forceinline__ float march_interior(const T *__restrict__ vol, const Ray &R)
{
    // ZB: the second transverse axis is z (stride 1), true unless m == z
    const Index sa = (Index)R.sa, sm = (Index)R.sm;
    const Index sb = ZB ? (Index)1 : (Index)R.sb;
    unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, R.j_lo, R.ic);
    unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, R.j_lo, R.ic);
    const unsigned long long ga = (unsigned long long)R.Ga, gb = (unsigned long long)R.Gb;
    Index plane = (Index)R.j_lo * sm;
    float acc = 0.0f;
    int i = R.j_lo;
    for (; i + kBatch - 1 <= R.j_hi; i += kBatch) {
        float v00[kBatch], v01[kBatch], v10[kBatch], v11[kBatch], da[kBatch], db[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            da[t] = frac_of(pa);
            db[t] = frac_of(pb);
            const T *p = vol + (plane + (Index)floor_of(pa) * sa + (Index)floor_of(pb) * sb);
            v00[t] = load_voxel(p);
            v01[t] = load_voxel(p + sb);
            v10[t] = load_voxel(p + sa);
            v11[t] = load_voxel(p + sa + sb);
            pa += ga;
            pb += gb;
            plane += sm;
        }
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            // Eq. 12 with w_lin (Eq. 13), as two nested linear interpolations
            const float e0 = __fmaf_rn(db[t], v01[t] - v00[t], v00[t]);
            const float e1 = __fmaf_rn(db[t], v11[t] - v10[t], v10[t]);
            acc += __fmaf_rn(da[t], e1 - e0, e0);
        }
    }
    for (; i <= R.j_hi; ++i) {
        const float da = frac_of(pa), db = frac_of(pb);
        const T *p = vol + (plane + (Index)floor_of(pa) * sa + (Index)floor_of(pb) * sb);
        const float v00 = load_voxel(p), v01 = load_voxel(p + sb);
        const float v10 = load_voxel(p + sa), v11 = load_voxel(p + sa + sb);
        const float e0 = __fmaf_rn(db, v01 - v00, v00);
        const float e1 = __fmaf_rn(db, v11 - v10, v10);
        acc += __fmaf_rn(da, e1 - e0, e0);
        pa += ga;
        pb += gb;
        plane += sm;
    }
    return acc;
}

template <typename T, typename Index>
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
        const float da = frac_of(pa), db = frac_of(pb);
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

template <typename T, typename Index>
__global__ void __launch_bounds__(kThreads) gjp_forward_kernel(
    const T *__restrict__ vol, VolParams V, const ViewParams *__restrict__ views,
    int nu, int nv, int n_tv, float *__restrict__ proj)
{
    const int tile = blockIdx.x;
    const int view = blockIdx.y;
    const int iv = (tile % n_tv) * kTileV + threadIdx.x;
    const int iu = (tile / n_tv) * kTileU + threadIdx.y;
    if (iv >= nv || iu >= nu) return;

    ViewParams vp;
    load_view(views, view, vp);
    Ray R;
    setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);

    float acc = (R.m != 2) ? march_interior<T, Index, true>(vol, R) : march_interior<T, Index, false>(vol, R);
    acc += march_boundary<T, Index>(vol, R);
    proj[((size_t)view * nv + iv) * nu + iu] = acc * R.step;
}

// ---------------------------------------------------------------------------
// Adjoint: the same (ray, plane, tap) triples scatter y * step * weight.

template <typename Index>
__global__ void __launch_bounds__(kThreads) gjp_adjoint_kernel(
    const float *__restrict__ proj, VolParams V, const ViewParams *__restrict__ views,
    int nu, int nv, int n_tv, float *__restrict__ vol)
{
    const int tile = blockIdx.x;
    const int view = blockIdx.y;
    const int iv = (tile % n_tv) * kTileV + threadIdx.x;
    const int iu = (tile / n_tv) * kTileU + threadIdx.y;
    if (iv >= nv || iu >= nu) return;
    const float y = __ldg(proj + ((size_t)view * nv + iv) * nu + iu);
    if (y == 0.0f) return;   // contributes exactly nothing

    ViewParams vp;
    load_view(views, view, vp);
    Ray R;
    setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);
    const float ys = y * R.step;
    const Index sa = (Index)R.sa, sb = (Index)R.sb, sm = (Index)R.sm;

    // interior planes
    unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, R.j_lo, R.ic);
    unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, R.j_lo, R.ic);
    Index plane = (Index)R.j_lo * sm;
    for (int i = R.j_lo; i <= R.j_hi; ++i) {
        const float da = frac_of(pa), db = frac_of(pb);
        float *p = vol + (plane + (Index)floor_of(pa) * sa + (Index)floor_of(pb) * sb);
        const float w0 = (1.0f - da) * ys, w1 = da * ys;
        atomicAdd(p, w0 * (1.0f - db));
        atomicAdd(p + sb, w0 * db);
        atomicAdd(p + sa, w1 * (1.0f - db));
        atomicAdd(p + sa + sb, w1 * db);
        pa += (unsigned long long)R.Ga;
        pb += (unsigned long long)R.Gb;
        plane += sm;
    }
    // boundary planes
    int n_before;
    const int nbd = boundary_count(R, n_before);
    const unsigned na = (unsigned)R.na, nb = (unsigned)R.nb;
    for (int k = 0; k < nbd; ++k) {
        const int i = boundary_plane(R, k, n_before);
        const unsigned long long qa = (unsigned long long)pos_at(R.Pa, R.Ga, i, R.ic);
        const unsigned long long qb = (unsigned long long)pos_at(R.Pb, R.Gb, i, R.ic);
        const float da = frac_of(qa), db = frac_of(qb);
        const int ia = floor_of(qa), ib = floor_of(qb);
        const bool a0 = (unsigned)ia < na, a1 = (unsigned)(ia + 1) < na;
        const bool b0 = (unsigned)ib < nb, b1 = (unsigned)(ib + 1) < nb;
        float *p = vol + ((Index)i * sm + (Index)ia * sa + (Index)ib * sb);
        const float w0 = (1.0f - da) * ys, w1 = da * ys;
        if (a0 && b0) atomicAdd(p, w0 * (1.0f - db));
        if (a0 && b1) atomicAdd(p + sb, w0 * db);
        if (a1 && b0) atomicAdd(p + sa, w1 * (1.0f - db));
        if (a1 && b1) atomicAdd(p + sa + sb, w1 * db);
    }
}

// Marks every voxel that receives a non-zero interpolation weight from a
// ray of one view (the view's compulsory volume traffic).
template <typename Index>
__global__ void __launch_bounds__(kThreads) gjp_footprint_kernel(
    VolParams V, const ViewParams *__restrict__ views, int view, int nu, int nv, int n_tv,
    unsigned char *__restrict__ marks)
{
    const int tile = blockIdx.x;
    const int iv = (tile % n_tv) * kTileV + threadIdx.x;
    const int iu = (tile / n_tv) * kTileU + threadIdx.y;
    if (iv >= nv || iu >= nu) return;
    ViewParams vp;
    load_view(views, view, vp);
    Ray R;
    setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);
    const Index sa = (Index)R.sa, sb = (Index)R.sb, sm = (Index)R.sm;
    const unsigned na = (unsigned)R.na, nb = (unsigned)R.nb;
    for (int i = R.s_lo; i <= R.s_hi; ++i) {
        const unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, i, R.ic);
        const unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, i, R.ic);
        const int ia = floor_of(pa), ib = floor_of(pb);
        const bool fa = (unsigned)pa != 0u, fb = (unsigned)pb != 0u;   // non-zero fraction
        const bool a0 = (unsigned)ia < na, a1 = (unsigned)(ia + 1) < na && fa;
        const bool b0 = (unsigned)ib < nb, b1 = (unsigned)(ib + 1) < nb && fb;
        unsigned char *p = marks + ((Index)i * sm + (Index)ia * sa + (Index)ib * sb);
        if (a0 && b0) p[0] = 1;
        if (a0 && b1) p[sb] = 1;
        if (a1 && b0) p[sa] = 1;
        if (a1 && b1) p[sa + sb] = 1;
    }
}

// ---------------------------------------------------------------------------
// Host helpers.

gjp_status check_grid(int64_t nx, int64_t ny, int64_t nz, const double h[3], const double *origin,
                      int64_t n[3], double hh[3], double o[3])
{
    if (nx < 1 || ny < 1 || nz < 1 || !h) return GJP_ERR_INVALID_ARG;
    if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30)) return GJP_ERR_INVALID_ARG;
    if ((double)nx * (double)ny * (double)nz > 9.0e18) return GJP_ERR_INVALID_ARG;
    n[0] = nx; n[1] = ny; n[2] = nz;
    for (int k = 0; k < 3; ++k) {
        if (!std::isfinite(h[k]) || !(h[k] > 0.0)) return GJP_ERR_INVALID_ARG;
        hh[k] = h[k];
        o[k] = origin ? origin[k] : -0.5 * (double)(n[k] - 1) * h[k];
        if (!std::isfinite(o[k])) return GJP_ERR_INVALID_ARG;
    }
    return GJP_OK;
}

// The whole line through the volume is integrated, which needs the source
// outside the support of the interpolated volume, (-1, n_k) in index units.
gjp_status check_sources(const gjp_geometry *g, const int64_t n[3], const double h[3], const double o[3])
{
    for (int k = 0; k < g->n_views; ++k) {
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
            const double s = (g->src[3 * k + a] - o[a]) / h[a];
            if (!(s > -1.0 && s < (double)n[a])) inside = false;
        }
        if (inside) return GJP_ERR_INVALID_ARG;
    }
    return GJP_OK;
}

VolParams make_vol(const int64_t n[3], const double h[3])
{
    VolParams V;
    for (int k = 0; k < 3; ++k) {
        V.n[k] = (int)n[k];
        V.h[k] = (float)h[k];
    }
    V.s[0] = (long long)(n[1] * n[2]);
    V.s[1] = (long long)n[2];
    V.s[2] = 1;
    return V;
}

bool fits_int32(const int64_t n[3])
{
    // every offset the loop forms (including out-of-range taps that are
    // masked) lies in [-(stride sum), nvox + stride sum]
    const double nvox = (double)n[0] * n[1] * n[2];
    return nvox + 2.0 * ((double)n[1] * n[2] + n[2] + 1) < 2147483647.0;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

const char *gjp_status_string(gjp_status s)
{
    switch (s) {
    case GJP_OK: return "GJP_OK";
    case GJP_ERR_INVALID_ARG: return "GJP_ERR_INVALID_ARG";
    case GJP_ERR_UNSUPPORTED: return "GJP_ERR_UNSUPPORTED";
    case GJP_ERR_OOM: return "GJP_ERR_OOM";
    case GJP_ERR_CUDA: return "GJP_ERR_CUDA";
    case GJP_ERR_INTERNAL: return "GJP_ERR_INTERNAL";
    case GJP_ERR_TIMEOUT: return "GJP_ERR_TIMEOUT";
    }
    return "GJP_ERR_UNKNOWN";
}

gjp_status gjp_geometry_create(int n_views, int nu, int nv, const double *src, const double *det_origin,
                               const double *det_u, const double *det_v, gjp_geometry **out)
{
    if (!out) return GJP_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_views < 1 || nu < 1 || nv < 1 || !src || !det_origin || !det_u || !det_v) return GJP_ERR_INVALID_ARG;
    if (nu > (1 << 24) || nv > (1 << 24) || n_views > (1 << 24)) return GJP_ERR_INVALID_ARG;
    for (int k = 0; k < n_views; ++k) {
        const double *s = src + 3 * k, *o = det_origin + 3 * k, *u = det_u + 3 * k, *v = det_v + 3 * k;
        if (!finite3(s) || !finite3(o) || !finite3(u) || !finite3(v)) return GJP_ERR_INVALID_ARG;
        const double nrm[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        const double nn = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        const double lu = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double lv = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(lu > 0.0) || !(lv > 0.0) || !(nn > 1e-12 * lu * lv)) return GJP_ERR_INVALID_ARG;
        // distance of the source from the detector plane
        const double dist = std::fabs(nrm[0] * (s[0] - o[0]) + nrm[1] * (s[1] - o[1]) + nrm[2] * (s[2] - o[2])) / nn;
        const double scale = std::sqrt((s[0] - o[0]) * (s[0] - o[0]) + (s[1] - o[1]) * (s[1] - o[1]) +
                                       (s[2] - o[2]) * (s[2] - o[2])) + lu + lv;
        if (!(dist > 1e-9 * scale)) return GJP_ERR_INVALID_ARG;
    }
    gjp_geometry *g = new (std::nothrow) gjp_geometry;
    if (!g) return GJP_ERR_OOM;
    try {
        g->n_views = n_views;
        g->nu = nu;
        g->nv = nv;
        g->src.assign(src, src + 3 * (size_t)n_views);
        g->org.assign(det_origin, det_origin + 3 * (size_t)n_views);
        g->du.assign(det_u, det_u + 3 * (size_t)n_views);
        g->dv.assign(det_v, det_v + 3 * (size_t)n_views);
    } catch (const std::bad_alloc &) {
        delete g;
        return GJP_ERR_OOM;
    }
    *out = g;
    return GJP_OK;
}

void gjp_geometry_destroy(gjp_geometry *g)
{
    if (!g) return;
    if (!g->cache.empty()) {   // only a geometry that was used on a device touches CUDA
        int cur = -1;
        const bool have_dev = cudaGetDevice(&cur) == cudaSuccess;
        for (auto &e : g->cache) {
            if (e.d_table) {
                cudaSetDevice(e.device);
                cudaFree(e.d_table);
            }
        }
        if (have_dev) cudaSetDevice(cur);
    }
    delete g;
}

gjp_status gjp_geometry_info(const gjp_geometry *g, int *n_views, int *nu, int *nv)
{
    if (!g) return GJP_ERR_INVALID_ARG;
    if (n_views) *n_views = g->n_views;
    if (nu) *nu = g->nu;
    if (nv) *nv = g->nv;
    return GJP_OK;
}

gjp_status gjp_forward(const void *d_volume, gjp_dtype dtype, int64_t nx, int64_t ny, int64_t nz,
                       const double voxel_size[3], const double volume_origin[3], const gjp_geometry *g,
                       float *d_proj, void *stream)
{
    if (!d_volume || !g || !d_proj) return GJP_ERR_INVALID_ARG;
    if (dtype != GJP_F32 && dtype != GJP_BF16 && dtype != GJP_F16) return GJP_ERR_INVALID_ARG;
    int64_t n[3];
    double h[3], o[3];
    gjp_status st = check_grid(nx, ny, nz, voxel_size, volume_origin, n, h, o);
    if (st != GJP_OK) return st;
    if ((st = check_sources(g, n, h, o)) != GJP_OK) return st;
    const ViewParams *table = nullptr;
    if ((st = get_table(g, n, h, o, &table)) != GJP_OK) return st;

    const VolParams V = make_vol(n, h);
    const int n_tv = (g->nv + kTileV - 1) / kTileV;
    const int n_tu = (g->nu + kTileU - 1) / kTileU;
    const dim3 grid((unsigned)(n_tv * n_tu), (unsigned)g->n_views);
    const dim3 block(kTileV, kTileU);
    cudaStream_t s = (cudaStream_t)stream;
    const bool i32 = fits_int32(n);
    if (grid.x > 2147483647u || g->n_views > 65535) return GJP_ERR_UNSUPPORTED;
    switch (dtype) {
    case GJP_F32:
        if (i32) gjp_forward_kernel<float, int><<<grid, block, 0, s>>>((const float *)d_volume, V, table, g->nu, g->nv, n_tv, d_proj);
        else gjp_forward_kernel<float, long long><<<grid, block, 0, s>>>((const float *)d_volume, V, table, g->nu, g->nv, n_tv, d_proj);
        break;
    case GJP_BF16:
        if (i32) gjp_forward_kernel<__nv_bfloat16, int><<<grid, block, 0, s>>>((const __nv_bfloat16 *)d_volume, V, table, g->nu, g->nv, n_tv, d_proj);
        else gjp_forward_kernel<__nv_bfloat16, long long><<<grid, block, 0, s>>>((const __nv_bfloat16 *)d_volume, V, table, g->nu, g->nv, n_tv, d_proj);
        break;
    case GJP_F16:
        if (i32) gjp_forward_kernel<__half, int><<<grid, block, 0, s>>>((const __half *)d_volume, V, table, g->nu, g->nv, n_tv, d_proj);
        else gjp_forward_kernel<__half, long long><<<grid, block, 0, s>>>((const __half *)d_volume, V, table, g->nu, g->nv, n_tv, d_proj);
        break;
    }
    return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

gjp_status gjp_adjoint(const float *d_proj, const gjp_geometry *g, int64_t nx, int64_t ny, int64_t nz,
                       const double voxel_size[3], const double volume_origin[3], float *d_volume,
                       int accumulate, void *stream)
{
    if (!d_volume || !g || !d_proj) return GJP_ERR_INVALID_ARG;
    int64_t n[3];
    double h[3], o[3];
    gjp_status st = check_grid(nx, ny, nz, voxel_size, volume_origin, n, h, o);
    if (st != GJP_OK) return st;
    if ((st = check_sources(g, n, h, o)) != GJP_OK) return st;
    const ViewParams *table = nullptr;
    if ((st = get_table(g, n, h, o, &table)) != GJP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!accumulate) {
        if (cudaMemsetAsync(d_volume, 0, sizeof(float) * (size_t)(n[0] * n[1] * n[2]), s) != cudaSuccess)
            return GJP_ERR_CUDA;
    }
    const VolParams V = make_vol(n, h);
    const int n_tv = (g->nv + kTileV - 1) / kTileV;
    const int n_tu = (g->nu + kTileU - 1) / kTileU;
    const dim3 grid((unsigned)(n_tv * n_tu), (unsigned)g->n_views);
    const dim3 block(kTileV, kTileU);
    if (g->n_views > 65535) return GJP_ERR_UNSUPPORTED;
    if (fits_int32(n)) gjp_adjoint_kernel<int><<<grid, block, 0, s>>>(d_proj, V, table, g->nu, g->nv, n_tv, d_volume);
    else gjp_adjoint_kernel<long long><<<grid, block, 0, s>>>(d_proj, V, table, g->nu, g->nv, n_tv, d_volume);
    return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

gjp_status gjp_footprint(const gjp_geometry *g, int view, int64_t nx, int64_t ny, int64_t nz,
                         const double voxel_size[3], const double volume_origin[3],
                         unsigned char *d_marks, void *stream)
{
    if (!g || !d_marks || view < 0 || view >= g->n_views) return GJP_ERR_INVALID_ARG;
    int64_t n[3];
    double h[3], o[3];
    gjp_status st = check_grid(nx, ny, nz, voxel_size, volume_origin, n, h, o);
    if (st != GJP_OK) return st;
    if ((st = check_sources(g, n, h, o)) != GJP_OK) return st;
    const ViewParams *table = nullptr;
    if ((st = get_table(g, n, h, o, &table)) != GJP_OK) return st;
    const VolParams V = make_vol(n, h);
    const int n_tv = (g->nv + kTileV - 1) / kTileV;
    const int n_tu = (g->nu + kTileU - 1) / kTileU;
    const dim3 grid((unsigned)(n_tv * n_tu));
    const dim3 block(kTileV, kTileU);
    cudaStream_t s = (cudaStream_t)stream;
    if (fits_int32(n)) gjp_footprint_kernel<int><<<grid, block, 0, s>>>(V, table, view, g->nu, g->nv, n_tv, d_marks);
    else gjp_footprint_kernel<long long><<<grid, block, 0, s>>>(V, table, view, g->nu, g->nv, n_tv, d_marks);
    return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

}  // extern "C"
