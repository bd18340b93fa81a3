// gjp.cu -- GB300 (sm_103a) branchless generalized Joseph projector:
// host-side geometry (FP64), forward and adjoint kernels, and the C ABI
// declared in include/gjp.h.
//
// Method: Algorithm 1 (Eq. 1-13) of Graetz, "High performance volume ray
// casting: A branchless generalized Joseph projector".  Each thread owns one
// ray (one detector pixel of one view), marches the integer planes
// perpendicular to its driving axis m and accumulates the bilinearly
// interpolated volume, scaled by the world length of one plane step.
//
// GB300 design points (see the repository's design notes for measurements):
//  * Per-view constants are formed in FP64 on the host and stored as FP32:
//    the ray direction r(u, v) = R0 + u RU + v RV and the moment of the ray
//    about the volume centre, L(u, v) = (s - c) x r.  The plane crossing at
//    the centre plane then follows from L / r_m without the catastrophic
//    cancellation of s + (o + i) rt with |s| ~ 3 volume widths, so a ray's
//    sample positions carry ~ulp(n) absolute error instead of ~ulp(|s|).
//  * The driving-axis coordinate of every sample is the plane index itself
//    (an exact integer, as Algorithm 1 asserts); the transverse positions
//    are one FMA from the plane index.
//  * The plane range of each ray is clipped in the setup to the planes that
//    can hold a non-zero tap; the clipped range is verified with the same
//    FMAs the loop uses (positions are monotone in the plane index), so the
//    clip never changes a result.
//  * Warps run along detector rows' neighbours in v, which map to the
//    contiguous z index of the volume: lanes of a warp read consecutive
//    voxels (the memory-order rule that accompanies Algorithm 1).
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
// Per-view device record: FP32 images of FP64 host quantities (index units,
// pixel coordinates centred on the panel: u = iu - (nu-1)/2, v = iv - (nv-1)/2).
struct ViewParams {
    float r0[3], ru[3], rv[3];  // ray direction d - s, Eq. 2, affine in (u, v)
    float m0[3], mu[3], mv[3];  // moment (s - c) x r about the volume centre c
};

struct VolParams {
    int n[3];
    float c[3];         // (n - 1) / 2
    float h[3];         // voxel size (world)
    long long s[3];     // element strides: ny*nz, nz, 1
};

constexpr int kTileV = 32;  // lanes of a warp along v (contiguous z)
constexpr int kTileU = 8;   // warps of a block along u
constexpr int kThreads = kTileV * kTileU;

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

// Host FP64 construction of the per-view table for one volume grid.
void build_table(const gjp_geometry &g, const int64_t n[3], const double h[3], const double o[3],
                 std::vector<ViewParams> &out)
{
    out.resize(g.n_views);
    const double cu = 0.5 * (g.nu - 1), cv = 0.5 * (g.nv - 1);
    for (int k = 0; k < g.n_views; ++k) {
        double s[3], R0[3], RU[3], RV[3];
        for (int a = 0; a < 3; ++a) {
            const double c = 0.5 * (double)(n[a] - 1);
            s[a] = (g.src[3 * k + a] - o[a]) / h[a] - c;                 // source, centred index units
            RU[a] = g.du[3 * k + a] / h[a];
            RV[a] = g.dv[3 * k + a] / h[a];
            R0[a] = (g.org[3 * k + a] - g.src[3 * k + a]) / h[a] + cu * RU[a] + cv * RV[a];
        }
        auto cross = [](const double *x, const double *y, double *z) {
            z[0] = x[1] * y[2] - x[2] * y[1];
            z[1] = x[2] * y[0] - x[0] * y[2];
            z[2] = x[0] * y[1] - x[1] * y[0];
        };
        double M0[3], MU[3], MV[3];
        cross(s, R0, M0);
        cross(s, RU, MU);
        cross(s, RV, MV);
        ViewParams &vp = out[k];
        for (int a = 0; a < 3; ++a) {
            vp.r0[a] = (float)R0[a];
            vp.ru[a] = (float)RU[a];
            vp.rv[a] = (float)RV[a];
            vp.m0[a] = (float)M0[a];
            vp.mu[a] = (float)MU[a];
            vp.mv[a] = (float)MV[a];
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
// Device side.

template <typename T> __device__ __forceinline__ float load_voxel(const T *p);
template <> __device__ __forceinline__ float load_voxel<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_voxel<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float load_voxel<__half>(const __half *p) { return __half2float(__ldg(p)); }

struct Ray {
    int m;            // driving axis (Eq. 3)
    int na, nb;       // transverse extents
    float Pa, Pb;     // transverse positions on the centre plane p_m = c_m
    float ga, gb;     // rt_a, rt_b (Eq. 4)
    float cm;         // c_m
    int i_lo, i_hi;   // clipped plane range (inclusive)
    float step;       // |h (.) rt|
    long long sm, sa, sb;
};

// Register select among three values (avoids local-memory arrays for
// indices known only at run time).
template <typename X> __device__ __forceinline__ X sel3(X x0, X x1, X x2, int k)
{
    return k == 0 ? x0 : (k == 1 ? x1 : x2);
}

// Plane i lies before (dir < 0) / after (dir > 0) the interval of planes
// with a possible non-zero tap, judged with the loop's own arithmetic.
__device__ __forceinline__ bool plane_beyond(float p, float g, int n, int dir)
{
    const float enter = (g > 0.0f) == (dir < 0) ? -1.0f : (float)n;  // bound crossed on that side
    if (g == 0.0f) return !(p > -1.0f && p < (float)n);
    if (enter < 0.0f) return p <= -1.0f;
    return p >= (float)n;
}

__device__ __forceinline__ bool range_side_ok(const Ray &R, int i, int dir)
{
    const float t = (float)i - R.cm;
    const float pa = fmaf(t, R.ga, R.Pa), pb = fmaf(t, R.gb, R.Pb);
    return plane_beyond(pa, R.ga, R.na, dir) || plane_beyond(pb, R.gb, R.nb, dir);
}

// Interval of t (= i - c_m) with -1 < P + t g < n, widened by `pad`.
__device__ __forceinline__ void t_bounds(float P, float g, int n, float &lo, float &hi)
{
    const float big = 3.0e7f;
    if (fabsf(g) < 1e-30f) {
        if (P > -1.0f && P < (float)n) { lo = -big; hi = big; }
        else { lo = big; hi = -big; }
        return;
    }
    float t0 = (-1.0f - P) / g, t1 = ((float)n - P) / g;
    lo = fmaxf(fminf(t0, t1), -big);
    hi = fminf(fmaxf(t0, t1), big);
}

__device__ __forceinline__ void setup_ray(const ViewParams &vp, const VolParams &V, float u, float v, Ray &R)
{
    const float r0 = fmaf(v, vp.rv[0], fmaf(u, vp.ru[0], vp.r0[0]));
    const float r1 = fmaf(v, vp.rv[1], fmaf(u, vp.ru[1], vp.r0[1]));
    const float r2 = fmaf(v, vp.rv[2], fmaf(u, vp.ru[2], vp.r0[2]));
    const float L0 = fmaf(v, vp.mv[0], fmaf(u, vp.mu[0], vp.m0[0]));
    const float L1 = fmaf(v, vp.mv[1], fmaf(u, vp.mu[1], vp.m0[1]));
    const float L2 = fmaf(v, vp.mv[2], fmaf(u, vp.mu[2], vp.m0[2]));
    int m = 0;                                   // Eq. 3, ties to the lowest index
    if (fabsf(r1) > fabsf(r0)) m = 1;
    if (fabsf(r2) > fabsf(sel3(r0, r1, r2, m))) m = 2;
    const int a = (m == 0) ? 1 : 0;
    const int b = (m == 2) ? 1 : 2;
    const float rm = sel3(r0, r1, r2, m);
    const float ra = sel3(r0, r1, r2, a), rb = sel3(r0, r1, r2, b);
    const float La = sel3(L0, L1, L2, a), Lb = sel3(L0, L1, L2, b);
    // crossing of the centre plane: q_k = (s_k r_m - s_m r_k) / r_m = +-L_j / r_m
    // (j the third axis; minus for the cyclic order (m, k, j))
    const float sgn_a = (a == (m + 1) % 3) ? -1.0f : 1.0f;
    const float sgn_b = (b == (m + 1) % 3) ? -1.0f : 1.0f;
    R.m = m;
    R.na = sel3(V.n[0], V.n[1], V.n[2], a);
    R.nb = sel3(V.n[0], V.n[1], V.n[2], b);
    R.Pa = sel3(V.c[0], V.c[1], V.c[2], a) + sgn_a * Lb / rm;
    R.Pb = sel3(V.c[0], V.c[1], V.c[2], b) + sgn_b * La / rm;
    R.ga = ra / rm;                              // Eq. 4
    R.gb = rb / rm;
    R.cm = sel3(V.c[0], V.c[1], V.c[2], m);
    const float hm = sel3(V.h[0], V.h[1], V.h[2], m);
    const float ha = sel3(V.h[0], V.h[1], V.h[2], a) * R.ga, hb = sel3(V.h[0], V.h[1], V.h[2], b) * R.gb;
    R.step = sqrtf(hm * hm + ha * ha + hb * hb);
    R.sm = sel3(V.s[0], V.s[1], V.s[2], m);
    R.sa = sel3(V.s[0], V.s[1], V.s[2], a);
    R.sb = sel3(V.s[0], V.s[1], V.s[2], b);

    // plane range: i in [0, n_m - 1] with -1 < p_k < n_k for both transverse k
    float lo_a, hi_a, lo_b, hi_b;
    t_bounds(R.Pa, R.ga, R.na, lo_a, hi_a);
    t_bounds(R.Pb, R.gb, R.nb, lo_b, hi_b);
    const float tlo = fmaxf(lo_a, lo_b), thi = fminf(hi_a, hi_b);
    const int nm = sel3(V.n[0], V.n[1], V.n[2], m);
    int i_lo = 0, i_hi = -1;
    if (tlo <= thi) {
        i_lo = max(0, (int)floorf(tlo + R.cm) - 1);
        i_hi = min(nm - 1, (int)ceilf(thi + R.cm) + 1);
    }
    // verify with the loop's arithmetic: the planes just outside the range
    // must lie beyond the support on their side; otherwise march everything
    bool ok = i_lo <= i_hi;
    if (ok && i_lo > 0) ok = range_side_ok(R, i_lo - 1, -1);
    if (ok && i_hi < nm - 1) ok = range_side_ok(R, i_hi + 1, +1);
    if (!ok) {
        // empty estimate: confirm emptiness cheaply at both ends, else full range
        bool empty = (i_lo > i_hi) && range_side_ok(R, nm - 1, -1);
        if (!empty) empty = (i_lo > i_hi) && range_side_ok(R, 0, +1);
        if (empty) { i_lo = 0; i_hi = -1; }
        else { i_lo = 0; i_hi = nm - 1; }
    }
    R.i_lo = i_lo;
    R.i_hi = i_hi;
}

__device__ __forceinline__ void load_view(const ViewParams *__restrict__ views, int k, ViewParams &vp)
{
    const float *src = reinterpret_cast<const float *>(views + k);
    float *dst = reinterpret_cast<float *>(&vp);
#pragma unroll
    for (int j = 0; j < 18; ++j) dst[j] = __ldg(src + j);
}

// One thread per ray; blockIdx.x = detector tile (v-tiles fastest), blockIdx.y = view.
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

    const Index sm = (Index)R.sm, sa = (Index)R.sa, sb = (Index)R.sb;
    const unsigned na = (unsigned)R.na, nb = (unsigned)R.nb;
    float acc = 0.0f;
    for (int i = R.i_lo; i <= R.i_hi; ++i) {
        const float t = (float)i - R.cm;
        const float pa = fmaf(t, R.ga, R.Pa);    // Eq. 6, transverse components
        const float pb = fmaf(t, R.gb, R.Pb);
        const float fa = floorf(pa), fb = floorf(pb);      // Eq. 7
        const float da = pa - fa, db = pb - fb;            // Eq. 10
        const int ia = (int)fa, ib = (int)fb;
        const bool a0 = (unsigned)ia < na, a1 = (unsigned)(ia + 1) < na;   // zero border
        const bool b0 = (unsigned)ib < nb, b1 = (unsigned)(ib + 1) < nb;
        const Index base = (Index)i * sm + (Index)ia * sa + (Index)ib * sb;
        const T *p = vol + base;
        const float v00 = (a0 && b0) ? load_voxel(p) : 0.0f;
        const float v01 = (a0 && b1) ? load_voxel(p + sb) : 0.0f;
        const float v10 = (a1 && b0) ? load_voxel(p + sa) : 0.0f;
        const float v11 = (a1 && b1) ? load_voxel(p + sa + sb) : 0.0f;
        // Eq. 12 with w_lin (Eq. 13): w_fl = 1 - d, w_cl = d
        const float wa0 = 1.0f - da, wb0 = 1.0f - db;
        acc += wa0 * (wb0 * v00 + db * v01) + da * (wb0 * v10 + db * v11);
    }
    proj[((size_t)view * nv + iv) * nu + iu] = acc * R.step;
}

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

    const Index sm = (Index)R.sm, sa = (Index)R.sa, sb = (Index)R.sb;
    const unsigned na = (unsigned)R.na, nb = (unsigned)R.nb;
    for (int i = R.i_lo; i <= R.i_hi; ++i) {
        const float t = (float)i - R.cm;
        const float pa = fmaf(t, R.ga, R.Pa);
        const float pb = fmaf(t, R.gb, R.Pb);
        const float fa = floorf(pa), fb = floorf(pb);
        const float da = pa - fa, db = pb - fb;
        const int ia = (int)fa, ib = (int)fb;
        const bool a0 = (unsigned)ia < na, a1 = (unsigned)(ia + 1) < na;
        const bool b0 = (unsigned)ib < nb, b1 = (unsigned)(ib + 1) < nb;
        const Index base = (Index)i * sm + (Index)ia * sa + (Index)ib * sb;
        float *p = vol + base;
        const float wa0 = (1.0f - da) * ys, wa1 = da * ys;
        const float wb0 = 1.0f - db;
        if (a0 && b0) atomicAdd(p, wa0 * wb0);
        if (a0 && b1) atomicAdd(p + sb, wa0 * db);
        if (a1 && b0) atomicAdd(p + sa, wa1 * wb0);
        if (a1 && b1) atomicAdd(p + sa + sb, wa1 * db);
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
    const Index sm = (Index)R.sm, sa = (Index)R.sa, sb = (Index)R.sb;
    const unsigned na = (unsigned)R.na, nb = (unsigned)R.nb;
    for (int i = R.i_lo; i <= R.i_hi; ++i) {
        const float t = (float)i - R.cm;
        const float pa = fmaf(t, R.ga, R.Pa);
        const float pb = fmaf(t, R.gb, R.Pb);
        const float fa = floorf(pa), fb = floorf(pb);
        const float da = pa - fa, db = pb - fb;
        const int ia = (int)fa, ib = (int)fb;
        const bool a0 = (unsigned)ia < na && da < 1.0f, a1 = (unsigned)(ia + 1) < na && da > 0.0f;
        const bool b0 = (unsigned)ib < nb && db < 1.0f, b1 = (unsigned)(ib + 1) < nb && db > 0.0f;
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
        V.c[k] = (float)(0.5 * (double)(n[k] - 1));
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
