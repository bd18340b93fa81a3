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
#include "gjp_common.cuh"

#include <atomic>

namespace gjp_detail {

bool finite3(const double *p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

std::atomic<int> g_fail_allocations{0};

bool alloc_gate()
{
    int n = g_fail_allocations.load();
    while (n > 0)
        if (g_fail_allocations.compare_exchange_weak(n, n - 1)) return false;
    return true;
}

// Stream-ordered workspace of the z-paired copy: one memory pool per
// device, owned by the library.  It keeps up to kPairsKeep bytes across
// synchronisations, so that repeated calls on grids up to that size reuse
// their memory instead of mapping it again; larger copies are returned to
// the device at the next synchronisation.
constexpr unsigned long long kPairsKeep = 8ull << 30;
std::mutex g_pairs_mu;
std::vector<std::pair<int, cudaMemPool_t>> g_pairs_pools;

cudaMemPool_t pairs_pool(int dev)
{
    std::lock_guard<std::mutex> lock(g_pairs_mu);
    for (const auto &p : g_pairs_pools)
        if (p.first == dev) return p.second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    unsigned long long keep = kPairsKeep;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pairs_pools.emplace_back(dev, pool);
    return pool;
}

// Whether AUTO's 16-bit forward reads a z-paired copy: 32 or more views
// and at least 2^27 view-voxels.  With few views the volume is read from
// DRAM about once and the copy only adds bytes (at 128^3 .. 512^3 it lost
// with 4 and 16 views and won with 64 and more); with little work the copy
// kernel and its allocation are not repaid (64^3 with 32 views: 30.6 vs
// 24.7 us, 128^3 with 32 views: 91.3 vs 90.2 us; 128^3 with 64 views and
// 192^3 with 32 won).
bool pairs_pay(int n_views, const int64_t n[3])
{
    return n_views >= 32 && (double)n_views * (double)n[0] * (double)n[1] * (double)n[2] >= 134217728.0;
}

// Allocates `bytes` on stream s for the z-paired copy.  GJP_ERR_UNSUPPORTED
// while s is being captured into a graph (the copy would become a graph
// allocation); GJP_ERR_OOM when the allocation gate refuses or the device
// has no room (the CUDA error is cleared).
gjp_status pairs_alloc(size_t bytes, cudaStream_t s, void **out)
{
    *out = nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return GJP_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return GJP_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GJP_ERR_CUDA;
    cudaMemPool_t pool = pairs_pool(dev);
    if (!pool) return GJP_ERR_CUDA;
    if (!alloc_gate()) return GJP_ERR_OOM;
    if (cudaMallocFromPoolAsync(out, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return GJP_ERR_OOM;
    }
    return GJP_OK;
}

void split(double x, float &hi, float &lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// Host FP64 setup of view k for one volume grid (Eq. 1-2 in index units):
// the ray direction r(u, v) = R0 + u RU + v RV from the source to the pixel
// centre at centred pixel coordinates (u, v), and its moment M = s x r
// about the volume centre, each split into hi + lo FP32 parts.
void make_view_params(const gjp_geometry &g, int k, const int64_t n[3], const double h[3], const double o[3],
                      ViewParams &vp)
{
    const double cu = 0.5 * (g.nu - 1), cv = 0.5 * (g.nv - 1);
    double s[3], R[9], M[9];
    for (int a = 0; a < 3; ++a) {
        const double c = 0.5 * (double)(n[a] - 1);
        s[a] = (g.src[3 * k + a] - o[a]) / h[a] - c;                         // source, centred index units
        R[3 + a] = g.du[3 * k + a] / h[a];
        R[6 + a] = g.dv[3 * k + a] / h[a];
        R[a] = (g.org[3 * k + a] - g.src[3 * k + a]) / h[a] + cu * R[3 + a] + cv * R[6 + a];
    }
    for (int t = 0; t < 3; ++t) {                                             // M = s x R (columns 0,1,2)
        const double *x = R + 3 * t;
        M[3 * t + 0] = s[1] * x[2] - s[2] * x[1];
        M[3 * t + 1] = s[2] * x[0] - s[0] * x[2];
        M[3 * t + 2] = s[0] * x[1] - s[1] * x[0];
    }
    for (int j = 0; j < 9; ++j) {
        split(R[j], vp.rh[j], vp.rl[j]);
        split(M[j], vp.mh[j], vp.ml[j]);
    }
}

// Median angle between the central rays (source to detector centre) of
// consecutive views: the rotation step of a circular scan (0 for one view).
double central_ray_step(const gjp_geometry &g)
{
    if (g.n_views < 2) return 0.0;
    std::vector<double> steps;
    steps.reserve(g.n_views - 1);
    double prev[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < g.n_views; ++k) {
        double d[3], nn = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double c = g.org[3 * k + a] + 0.5 * (g.nu - 1) * g.du[3 * k + a] + 0.5 * (g.nv - 1) * g.dv[3 * k + a];
            d[a] = c - g.src[3 * k + a];
            nn += d[a] * d[a];
        }
        nn = std::sqrt(nn);
        for (int a = 0; a < 3; ++a) d[a] /= nn;
        if (k > 0) {
            const double cx = prev[1] * d[2] - prev[2] * d[1], cy = prev[2] * d[0] - prev[0] * d[2],
                         cz = prev[0] * d[1] - prev[1] * d[0];
            const double dot = prev[0] * d[0] + prev[1] * d[1] + prev[2] * d[2];
            steps.push_back(std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz), dot));
        }
        for (int a = 0; a < 3; ++a) prev[a] = d[a];
    }
    std::nth_element(steps.begin(), steps.begin() + steps.size() / 2, steps.end());
    return steps[steps.size() / 2];
}

// Host FP64 construction of the per-view table for one volume grid.
void build_table(const gjp_geometry &g, const int64_t n[3], const double h[3], const double o[3],
                 std::vector<ViewParams> &out)
{
    out.resize(g.n_views);
    for (int k = 0; k < g.n_views; ++k) make_view_params(g, k, n, h, o, out[k]);
}

// Returns the cache entry (device table) for (g, current device, grid);
// builds it on first use.
gjp_status get_table(const gjp_geometry *gc, const int64_t n[3], const double h[3], const double o[3],
                     gjp_cache_entry **out)
{
    gjp_geometry *g = const_cast<gjp_geometry *>(gc);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GJP_ERR_CUDA;
    double key[9] = {(double)n[0], (double)n[1], (double)n[2], h[0], h[1], h[2], o[0], o[1], o[2]};
    std::lock_guard<std::mutex> lock(g->mu);
    for (auto &e : g->cache) {
        if (e.device == dev && std::memcmp(e.key, key, sizeof key) == 0) {
            *out = &e;
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
    if (!alloc_gate() || cudaMalloc(&d, bytes) != cudaSuccess) {
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
    e.box_rows = e.box_cols4 = e.box_cols8 = 0;
    try {
        g->cache.push_back(e);
    } catch (const std::bad_alloc &) {
        cudaFree(d);
        return GJP_ERR_OOM;
    }
    *out = &g->cache.back();
    return GJP_OK;
}

template <typename T, typename Index, bool SPL, bool PAIRS>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocksMax) gjp_forward_kernel(
    const T *__restrict__ vol, VolParams V, const ViewParams *__restrict__ views,
    int nu, int nv, int n_tv, int n_views, int view_group, float *__restrict__ proj,
    const typename PairOf<T>::type *__restrict__ pairs)
{
    int tile, view;
    block_tile_view(n_views, view_group, tile, view);
    const int iv = (tile % n_tv) * kTileV + threadIdx.x;
    const int iu = (tile / n_tv) * (int)blockDim.y + threadIdx.y;
    const unsigned act = __ballot_sync(0xffffffffu, iv < nv && iu < nu);
    if (iv >= nv || iu >= nu) return;
    proj[((size_t)view * nv + iv) * nu + iu] =
        forward_ray<T, Index, SPL, PAIRS>(vol, V, views + view, nu, nv, iu, iv, act, (int)threadIdx.y, pairs);
}

// The z-paired copy of a 16-bit volume whose z lines are whole 8-byte words
// (nz % 4 == 0, 8-byte aligned base): a thread reads four voxels with one
// 8-byte load plus the next line voxel and writes their four pair words with
// one 16-byte store.
__global__ void gjp_zpairs16x4_kernel(const unsigned short *__restrict__ vol, long long lines, int nz,
                                      uint4 *__restrict__ out)
{
    const int quads = nz >> 2;
    for (long long r = blockIdx.x; r < lines; r += gridDim.x) {
        const unsigned short *line = vol + r * nz;
        const uint2 *src = reinterpret_cast<const uint2 *>(line);
        uint4 *o = out + r * quads;
        for (int k = threadIdx.x; k < quads; k += blockDim.x) {
            const uint2 w = __ldg(src + k);                              // voxels 4k .. 4k + 3
            const unsigned next = 4 * k + 4 < nz ? (unsigned)__ldg(line + 4 * k + 4) : 0u;
            o[k] = make_uint4(w.x, __funnelshift_r(w.x, w.y, 16), w.y, (w.y >> 16) | (next << 16));
        }
    }
}

// The z-paired copy of a volume (read by the row-table march): element e
// holds voxels e and e + 1 of its z line, the upper one zero at the last z.
// One block per z line at a time; consecutive threads take consecutive z.
template <typename T>
__global__ void gjp_zpairs_kernel(const T *__restrict__ vol, long long lines, int nz,
                                  typename PairOf<T>::type *__restrict__ out)
{
    using W = typename Raw<T>::type;
    for (long long r = blockIdx.x; r < lines; r += gridDim.x) {
        const T *line = vol + r * nz;
        typename PairOf<T>::type *o = out + r * nz;
        for (int z = threadIdx.x; z < nz; z += blockDim.x) {
            const W lo = load_raw(line + z), hi = z + 1 < nz ? load_raw(line + z + 1) : W(0);
            if constexpr (std::is_same<T, float>::value)
                o[z] = make_float2(lo, hi);
            else
                o[z] = (unsigned)lo | ((unsigned)hi << 16);
        }
    }
}

// ---------------------------------------------------------------------------
// Forward projection, shared-memory slab pipeline.
//
// A block owns a tile of kSlabWarps detector columns x 32 detector rows.
// When every ray of the tile shares its driving axis (x or y), the rays
// advance through the same sequence of planes.  The planes are taken
// kPlanes at a time (a "stage"): the producer warp computes, from the
// tile's four corner rays at the stage's first and last plane (a plane's
// crossings are a projective image of the tile, so their extremes sit at the
// corners, and each ray moves linearly from plane to plane), the box of
// voxels the stage's taps can touch, and one TMA tensor load brings that
// kPlanes x rows x cols box into a ring of shared-memory stages.  The
// consumer warps read their taps from shared memory.  Out-of-range parts of
// a box are zero-filled by the TMA unit, which is exactly the zero-border
// reading of "p is in volume".  Stages whose box would not fit, and tiles
// with mixed driving axes, use the global-memory gather above.

constexpr int kSlabWarps = 8;
constexpr int kSlabThreads = (kSlabWarps + 1) * 32;
constexpr int kStages = 4;       // ring depth
constexpr int kPlanes = 4;       // planes per stage
constexpr int kBoxRMax = 24;     // largest box extent along the non-contiguous transverse axis
constexpr unsigned kSpinLimit = 1u << 22;

// Set by a kernel whose bounded wait gave up; read and cleared by
// gjp_stream_status().
__device__ unsigned g_gjp_status;

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: false (and the status word set) if the phase has not
// completed after kSpinLimit polls or kWaitLimitNs of wall time, whichever
// comes first (try_wait may suspend the thread between polls for a
// hardware-defined time, so the clock bounds the wait, not the count).
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    const unsigned long long t0 = global_ns();
    for (unsigned spin = 0; spin < kSpinLimit; ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) break;
    }
    atomicOr(&g_gjp_status, 1u);
    return false;
}

// Failure-detection self-test: one thread waits, through the same bounded
// wait as the pipelines, on an mbarrier phase that nothing completes (the
// barrier expects one arrival and none comes).  The wait gives up after its
// limit, sets the status word and the kernel returns; no memory other than
// its own shared word is touched.
// Debug build: one thread records a tap outside the grid through the same
// check as the marches (indices only; nothing is accessed).
__global__ void gjp_tap_check_selftest_kernel() { taps_in_grid(-1, 0, 0, 1, 2, 2); }

__global__ void gjp_wait_selftest_kernel()
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_wait(&bar, 0);
    }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, unsigned long long *bar, int c0,
                                            int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_addr(bar)), "r"(c0),
        "r"(c1), "r"(c2)
        : "memory");
}

struct SlabShared {
    unsigned long long full[kStages], empty[kStages];
    int4 hdr[kStages];              // a0, b0, box fits, unused
    long long corner[4][4];         // Pa, Ga, Pb, Gb of the tile's corner rays
    int sweep_lo, sweep_hi, m_first, mixed;
};

template <typename T, typename Index, int kBoxC>
__global__ void __launch_bounds__(kSlabThreads, GJP_SLAB_MIN_BLOCKS) gjp_forward_slab_kernel(
    const T *__restrict__ vol, VolParams V, const ViewParams *__restrict__ views, int nu, int nv, int n_tv,
    int n_views, int view_group, const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_y,
    int box_r, float *__restrict__ proj)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int kAlign = 16 / (int)sizeof(T);               // TMA x coordinate granularity
    const int stage_elems = kPlanes * box_r * kBoxC;
    const int stage_bytes = (stage_elems * (int)sizeof(T) + 127) & ~127;
    SlabShared &S = *reinterpret_cast<SlabShared *>(smem_raw + kStages * stage_bytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp == kSlabWarps;
    int tile, view;
    block_tile_view(n_views, view_group, tile, view);
    const int v_base = (tile % n_tv) * 32, u_base = (tile / n_tv) * kSlabWarps;
    const int iv = v_base + lane, iu = u_base + warp;
    const bool have_ray = !producer && iv < nv && iu < nu;

    if (threadIdx.x == 0) {
        S.sweep_lo = 0x7fffffff;
        S.sweep_hi = -1;
        S.m_first = -1;
        S.mixed = 0;
        for (int k = 0; k < kStages; ++k) {
            mbar_init(&S.full[k], 1);
            mbar_init(&S.empty[k], kSlabWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    Ray R;
    if (have_ray) {
        ViewParams vp;
        load_view(views, view, vp);
        setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);
        if (R.s_lo <= R.s_hi) {
            atomicMin(&S.sweep_lo, R.s_lo);
            atomicMax(&S.sweep_hi, R.s_hi);
        }
        atomicCAS(&S.m_first, -1, R.m);
    }
    __syncthreads();
    if (have_ray) {
        if (R.m != S.m_first) S.mixed = 1;
        const int u_last = min(kSlabWarps, nu - u_base) - 1, v_last = min(32, nv - v_base) - 1;
        // a thread may be several corners when the tile is one ray wide
        for (int cu = 0; cu < 2; ++cu)
            for (int cv = 0; cv < 2; ++cv)
                if ((cu == 0 ? warp == 0 : warp == u_last) && (cv == 0 ? lane == 0 : lane == v_last)) {
                    long long *c = S.corner[2 * cu + cv];
                    c[0] = R.Pa;
                    c[1] = R.Ga;
                    c[2] = R.Pb;
                    c[3] = R.Gb;
                }
    }
    __syncthreads();

    const int m = S.m_first;
    if (S.mixed || m < 0 || m == 2) {       // gather path for the whole tile
        if (have_ray) {
            float acc = (R.m != 2) ? march_interior<T, Index, true>(vol, R) : march_interior<T, Index, false>(vol, R);
            acc += march_boundary<T, Index>(vol, R);
            proj[((size_t)view * nv + iv) * nu + iu] = acc * R.step;
        }
        return;
    }
    const int I0 = S.sweep_lo, I1 = S.sweep_hi;
    const int n_stages = I1 >= I0 ? (I1 - I0) / kPlanes + 1 : 0;
    T *stages = reinterpret_cast<T *>(smem_raw);
    const int stage_stride = stage_bytes / (int)sizeof(T);
    // shared-memory layout of a box: plane x = i boxes are [plane][row][col],
    // plane y = i boxes are [row][plane][col] (TMA writes dimension 0 fastest)
    const int row_stride = m == 0 ? kBoxC : kPlanes * kBoxC;
    const int plane_stride = m == 0 ? box_r * kBoxC : kBoxC;

    if (producer) {
        const int nm = V.n[m];
        const int ic = (nm - 1) >> 1;
        const unsigned tx = (unsigned)(stage_elems * (int)sizeof(T));
        // lane l tracks corner l & 3 at the stage's first (l < 4) or last plane
        const long long *cr = S.corner[lane & 3];
        const long long Pa = cr[0], Ga = cr[1], Pb = cr[2], Gb = cr[3];
        const int end = (lane >> 2) & 1;
        int slot = 0;
        unsigned phase = 0;
        bool ok = true;
        int st = 0;
        for (; st < n_stages; ++st) {
            if (st >= kStages) ok = mbar_wait(&S.empty[slot], phase ^ 1u);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            const int i0 = I0 + st * kPlanes;
            const int i = end ? min(i0 + kPlanes - 1, I1) : i0;
            const int fa = floor_of((unsigned long long)pos_at(Pa, Ga, i, ic));
            const int fb = floor_of((unsigned long long)pos_at(Pb, Gb, i, ic));
            const int amin = __reduce_min_sync(0xffffffffu, fa), amax = __reduce_max_sync(0xffffffffu, fa);
            const int bmin = __reduce_min_sync(0xffffffffu, fb), bmax = __reduce_max_sync(0xffffffffu, fb);
            if (lane == 0) {
                // one voxel of margin below, taps reach floor + 1, one voxel of margin above
                const int a0 = amin - 1;
                const int b0 = (bmin - 1) & ~(kAlign - 1);
                const bool fits = (amax + 3 - a0 <= box_r) && (bmax + 3 - b0 <= kBoxC);
                S.hdr[slot] = make_int4(a0, b0, fits ? 1 : 0, 0);
                if (fits) {
                    mbar_arrive_expect_tx(&S.full[slot], tx);
                    T *dst = stages + slot * stage_stride;
                    if (m == 0) tma_load_3d(dst, &map_x, &S.full[slot], b0, a0, i0);   // planes x = i0 ..
                    else tma_load_3d(dst, &map_y, &S.full[slot], b0, i0, a0);          // planes y = i0 ..
                } else {
                    mbar_arrive(&S.full[slot]);
                }
            }
            if (++slot == kStages) {
                slot = 0;
                phase ^= 1u;
            }
        }
        if (!ok && lane == 0) {
            // a consumer stopped; wait (bounded) for the copies still in flight
            for (int k = 0; k < kStages && k < st; ++k) {
                if (--slot < 0) {
                    slot = kStages - 1;
                    phase ^= 1u;
                }
                mbar_wait(&S.full[slot], phase);
            }
        }
        return;
    }

    // consumers
    const unsigned na = have_ray ? (unsigned)R.na : 0u, nb = have_ray ? (unsigned)R.nb : 0u;
    const Index sa = have_ray ? (Index)R.sa : 0, sb = have_ray ? (Index)R.sb : 0, sm = have_ray ? (Index)R.sm : 0;
    unsigned long long pa = 0, pb = 0, ga = 0, gb = 0;
    int s_lo = 1, s_hi = 0;
    if (have_ray) {
        pa = (unsigned long long)pos_at(R.Pa, R.Ga, I0, R.ic);
        pb = (unsigned long long)pos_at(R.Pb, R.Gb, I0, R.ic);
        ga = (unsigned long long)R.Ga;
        gb = (unsigned long long)R.Gb;
        s_lo = R.s_lo;
        s_hi = R.s_hi;
    }
    const unsigned max_idx = (unsigned)(stage_elems - row_stride - 2);
    float acc = 0.0f;
    int slot = 0;
    unsigned phase = 0;
    bool ok = true;
    for (int st = 0; st < n_stages; ++st) {
        if (ok) ok = mbar_wait(&S.full[slot], phase);
        const int4 h = S.hdr[slot];
        const T *box = stages + slot * stage_stride;
        const int i0 = I0 + st * kPlanes;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const int i = i0 + p;
            if (ok && i >= s_lo && i <= s_hi) {
                const float da = frac_of(pa), db = frac_of(pb);
                const int ia = floor_of(pa), ib = floor_of(pb);
                float v00, v01, v10, v11;
                if (h.z) {
                    // taps lie in the box by construction; the unsigned min only
                    // guards the shared-memory bounds
                    const unsigned idx = min((unsigned)((ia - h.x) * row_stride + (ib - h.y) + p * plane_stride),
                                             max_idx);
                    const T *s = box + idx;
                    v00 = to_float(s[0]);
                    v01 = to_float(s[1]);
                    v10 = to_float(s[row_stride]);
                    v11 = to_float(s[row_stride + 1]);
                } else {
                    const bool a0 = (unsigned)ia < na, a1 = (unsigned)(ia + 1) < na;
                    const bool b0 = (unsigned)ib < nb, b1 = (unsigned)(ib + 1) < nb;
                    const T *q = vol + ((Index)i * sm + (Index)ia * sa + (Index)ib * sb);
                    v00 = (a0 && b0) ? load_voxel(q) : 0.0f;
                    v01 = (a0 && b1) ? load_voxel(q + sb) : 0.0f;
                    v10 = (a1 && b0) ? load_voxel(q + sa) : 0.0f;
                    v11 = (a1 && b1) ? load_voxel(q + sa + sb) : 0.0f;
                }
                const float e0 = __fmaf_rn(db, v01 - v00, v00);
                const float e1 = __fmaf_rn(db, v11 - v10, v10);
                acc += __fmaf_rn(da, e1 - e0, e0);
            }
            pa += ga;
            pb += gb;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[slot]);
        if (++slot == kStages) {
            slot = 0;
            phase ^= 1u;
        }
    }
    if (have_ray) proj[((size_t)view * nv + iv) * nu + iu] = acc * R.step;
}

// ---------------------------------------------------------------------------
// Forward projection, gather with L2 prefetch: the gather kernel above, in
// which one lane per warp asks the TMA unit to bring the warp's footprint
// for planes kPfDist ahead (a box of kPfRows rows x kPlanes planes x
// kPfCols elements around the lane's own ray) from DRAM into L2, so the
// warp's later tap loads hit L2 instead of DRAM.

constexpr int kPfDist = 8;
constexpr int kPfRows = 4;

__device__ __forceinline__ void tma_prefetch_l2_3d(const CUtensorMap *map, int c0, int c1, int c2)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<unsigned long long>(map)),
                 "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

template <typename T, typename Index, bool ZB>
__device__ __forceinline__ float march_interior_pf(const T *__restrict__ vol, const Ray &R, bool leader,
                                                   const CUtensorMap *map)
{
    constexpr int kAlign = 16 / (int)sizeof(T);
    const Index sa = (Index)R.sa, sm = (Index)R.sm;
    const Index sb = ZB ? (Index)1 : (Index)R.sb;
    unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, R.j_lo, R.ic);
    unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, R.j_lo, R.ic);
    const unsigned long long ga = (unsigned long long)R.Ga, gb = (unsigned long long)R.Gb;
    const unsigned long long da_pf = ga * (unsigned long long)kPfDist, db_pf = gb * (unsigned long long)kPfDist;
    const unsigned long long da_span = ga * (unsigned long long)(kPlanes - 1), db_span = gb * (unsigned long long)(kPlanes - 1);
    Index plane = (Index)R.j_lo * sm;
    // two-level sum: planes of a batch are added together, batch sums are
    // folded into a partial sum that joins the total every 4 batches, so the
    // total sees one addition per 16 planes (float32 error ~4x smaller than
    // a running sum over up to ~n_m planes)
    float acc = 0.0f, part = 0.0f;
    int nb = 0;
    int i = R.j_lo;
    for (; i + kBatch - 1 <= R.j_hi; i += kBatch) {
        if (leader && i + kPfDist <= R.j_hi) {
            const unsigned long long qa = pa + da_pf, qb = pb + db_pf;
            const int a0 = min(floor_of(qa), floor_of(qa + da_span));
            const int b0 = (min(floor_of(qb), floor_of(qb + db_span)) - 1) & ~(kAlign - 1);
            if (R.m == 0) tma_prefetch_l2_3d(map, b0, a0, i + kPfDist);
            else tma_prefetch_l2_3d(map, b0, i + kPfDist, a0);
        }
        float v00[kBatch], v01[kBatch], v10[kBatch], v11[kBatch], da[kBatch], db[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            da[t] = frac_of(pa);
            db[t] = frac_of(pb);
            const bool ok = taps_in_grid(i + t, floor_of(pa), floor_of(pb), R.nm, R.na, R.nb);   // debug build only
            const T *p = vol + (plane + (Index)floor_of(pa) * sa + (Index)floor_of(pb) * sb);
            v00[t] = ok ? load_voxel(p) : 0.0f;
            v01[t] = ok ? load_voxel(p + sb) : 0.0f;
            v10[t] = ok ? load_voxel(p + sa) : 0.0f;
            v11[t] = ok ? load_voxel(p + sa + sb) : 0.0f;
            pa += ga;
            pb += gb;
            plane += sm;
        }
        float bsum = 0.0f;
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            // Eq. 12 with the weights of Eq. 13/14, as two nested interpolations
            const float e0 = __fmaf_rn(db[t], v01[t] - v00[t], v00[t]);
            const float e1 = __fmaf_rn(db[t], v11[t] - v10[t], v10[t]);
            bsum += __fmaf_rn(da[t], e1 - e0, e0);
        }
        part += bsum;
        if ((++nb & 3) == 0) {
            acc += part;
            part = 0.0f;
        }
    }
    acc += part;
    for (; i <= R.j_hi; ++i) {
        const float da = frac_of(pa), db = frac_of(pb);
        const bool ok = taps_in_grid(i, floor_of(pa), floor_of(pb), R.nm, R.na, R.nb);
        const T *p = vol + (plane + (Index)floor_of(pa) * sa + (Index)floor_of(pb) * sb);
        const float v00 = ok ? load_voxel(p) : 0.0f, v01 = ok ? load_voxel(p + sb) : 0.0f;
        const float v10 = ok ? load_voxel(p + sa) : 0.0f, v11 = ok ? load_voxel(p + sa + sb) : 0.0f;
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
__global__ void __launch_bounds__(kMaxThreads, kMinBlocksMax) gjp_forward_pf_kernel(
    const T *__restrict__ vol, VolParams V, const ViewParams *__restrict__ views, int nu, int nv, int n_tv,
    int n_views, int view_group, const __grid_constant__ CUtensorMap pf_map, float *__restrict__ proj)
{
    int tile, view;
    block_tile_view(n_views, view_group, tile, view);
    const int iv = (tile % n_tv) * kTileV + threadIdx.x;
    const int iu = (tile / n_tv) * (int)blockDim.y + threadIdx.y;
    if (iv >= nv || iu >= nu) return;

    ViewParams vp;
    load_view(views, view, vp);
    Ray R;
    setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);

    const bool leader = threadIdx.x == 0;   // lowest v of the warp: lowest z of its footprint
    float acc = (R.m != 2) ? march_interior_pf<T, Index, true>(vol, R, leader, &pf_map)
                           : march_interior<T, Index, false>(vol, R);
    acc += march_boundary<T, Index>(vol, R);
    proj[((size_t)view * nv + iv) * nu + iu] = acc * R.step;
}

// ---------------------------------------------------------------------------
// Adjoint: the same (ray, plane, tap) triples scatter y * step * weight.

// Scatter of one ray over all its planes with global float atomics.
template <typename Index, bool SPL = false>
__device__ __forceinline__ void scatter_ray(const Ray &R, float ys, float *__restrict__ vol)
{
    const Index sa = (Index)R.sa, sb = (Index)R.sb, sm = (Index)R.sm;
    // interior planes
    unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, R.j_lo, R.ic);
    unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, R.j_lo, R.ic);
    Index plane = (Index)R.j_lo * sm;
    for (int i = R.j_lo; i <= R.j_hi; ++i) {
        const float da = upper_weight<SPL>(frac_of(pa)), db = upper_weight<SPL>(frac_of(pb));
        float *p = vol + (plane + (Index)floor_of(pa) * sa + (Index)floor_of(pb) * sb);
        const float w0 = (1.0f - da) * ys, w1 = da * ys;
        if (taps_in_grid(i, floor_of(pa), floor_of(pb), R.nm, R.na, R.nb)) {   // always true but in the debug build
            atomicAdd(p, w0 * (1.0f - db));
            atomicAdd(p + sb, w0 * db);
            atomicAdd(p + sa, w1 * (1.0f - db));
            atomicAdd(p + sa + sb, w1 * db);
        }
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
        const float da = upper_weight<SPL>(frac_of(qa)), db = upper_weight<SPL>(frac_of(qb));
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

template <typename Index, bool SPL>
__global__ void __launch_bounds__(kMaxThreads) gjp_adjoint_kernel(
    const float *__restrict__ proj, VolParams V, const ViewParams *__restrict__ views,
    int nu, int nv, int n_tv, int n_views, int view_group, float *__restrict__ vol)
{
    int tile, view;
    block_tile_view(n_views, view_group, tile, view);
    const int iv = (tile % n_tv) * kTileV + threadIdx.x;
    const int iu = (tile / n_tv) * (int)blockDim.y + threadIdx.y;
    if (iv >= nv || iu >= nu) return;
    const float y = __ldg(proj + ((size_t)view * nv + iv) * nu + iu);
    if (y == 0.0f) return;   // contributes exactly nothing

    ViewParams vp;
    load_view(views, view, vp);
    Ray R;
    setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);
    scatter_ray<Index, SPL>(R, y * R.step, vol);
}

// ---------------------------------------------------------------------------
// Adjoint, warp-combined scatter.
//
// The transpose scatters four taps per sample.  Where all 32 rays of a warp
// (one detector column, 32 consecutive rows) share the driving axis m != z
// and their transverse position and increment along the other non-z axis a
// -- which holds bit for bit for a circular orbit about z with detector
// rows along z, because a ray's (x, y) path does not depend on its row --
// every sample of the warp at plane i lands in the same two rows a = ia and
// ia + 1, weighted 1 - da and da with one da for the whole warp.  The warp
// then marches its planes in step, and per plane a lane's upper z tap
// (ib + 1, weight ys db) usually is the next lane's lower tap: one shuffle
// hands it over, and the next lane adds both with a single reduction per
// row.  A lane whose upper tap is not the next lane's lower tap (a gap, two
// rays on one voxel, or the warp's last lane) adds it itself, so the result
// does not depend on how the rays are spaced.  This halves the reductions
// of the tap-by-tap scatter.  Warps without a common row scatter tap by tap.

// Reductions at p0 and p1 when w is set.  (The branch form measured faster
// than reductions predicated in the instruction, which also made the
// compiler emit more branches around them.)
__device__ __forceinline__ void red_add2_if(bool w, float *p0, float v0, float *p1, float v1)
{
    if (w) {
        atomicAdd(p0, v0);
        atomicAdd(p1, v1);
    }
}

__device__ __forceinline__ void red_add_if(bool w, float *p, float v)
{
    if (w) atomicAdd(p, v);
}

// What one lane adds to voxels ib (x0, when w0) and ib + 1 (x1, when w1) of
// both rows, given its taps g0 (to ib) and g1 (to ib + 1); see above.  ASC:
// the warp's z indices ascend with the lane index (else they descend, as for
// detector rows along -z); the run form walks the lanes in z order.
template <bool RUNS, bool ASC>
__device__ __forceinline__ void combine_lane(int ib, float g0, float g1, float &x0, float &x1, bool &w0, bool &w1)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x;
    if (RUNS) {
        // At most two neighbouring lanes share a voxel (checked once per
        // warp).  A run is one lane or two lanes on one voxel; its first lane
        // (in z order) adds the run's lower taps plus, when the previous
        // run's voxel is the one just below, that run's upper taps; a run's
        // last lane adds the run's upper taps itself only when no next run
        // starts on that voxel.  Every voxel then has one writer.
        // the z-previous and z-next lanes (a lane at the warp's end gets its
        // own value back, which the has_prev / has_next tests then ignore)
        const auto from_prev = [full](auto v) { return ASC ? __shfl_up_sync(full, v, 1) : __shfl_down_sync(full, v, 1); };
        const auto from_next = [full](auto v) { return ASC ? __shfl_down_sync(full, v, 1) : __shfl_up_sync(full, v, 1); };
        const bool has_prev = ASC ? lane > 0 : lane < 31, has_next = ASC ? lane < 31 : lane > 0;
        const int ib_p = from_prev(ib);
        const float g1_p = from_prev(g1);
        const int ib_n = from_next(ib);
        const int dn = has_next ? ib_n - ib : 2;      // z-last lane: no next run
        const int up = has_prev ? ib - ib_p : 2;      // z-first lane: no previous run
        const float g0_n = from_next(g0);
        const float e1 = up == 0 ? g1 + g1_p : g1;    // the run's upper taps, at its last lane
        const float e1_p = from_prev(e1);
        const float s0 = dn == 0 ? g0 + g0_n : g0;    // the run's lower taps, at its first lane
        x0 = up == 1 ? s0 + e1_p : s0;
        x1 = e1;
        w0 = up != 0;                                 // first lane of its run
        w1 = (unsigned)dn > 1u;                       // last lane, and no next run on voxel ib + 1
    } else {
        // the previous lane's upper tap joins this lane's lower tap when they
        // are the same voxel (lane 0 receives its own values: never taken)
        const int ib_up = __shfl_up_sync(full, ib, 1);
        const float g1_up = __shfl_up_sync(full, g1, 1);
        const int ib_dn = __shfl_down_sync(full, ib, 1);
        x0 = ib_up + 1 == ib ? g0 + g1_up : g0;
        x1 = g1;
        w0 = x0 != 0.0f;
        w1 = ib_dn != ib + 1 && g1 != 0.0f;          // kept when the next lane does not take it
    }
}

// One plane of the warp-combined adjoint (see above).  CHECKED tests each
// tap against the grid (zero border) and, with CLIP, the plane against the
// ray's clipped support; unchecked planes are interior for every lane.
template <typename Index, bool SPL, bool CHECKED, bool CLIP, bool RUNS, bool ASC>
__device__ __forceinline__ void combine_plane(const Ray &R, int i, float yw, unsigned long long &pa,
                                              unsigned long long &pb, Index &plane, Index sa, unsigned na,
                                              unsigned nb, float *__restrict__ vol)
{
    const int ia = floor_of(pa), ib = floor_of(pb);
    const float da = upper_weight<SPL>(frac_of(pa)), db = upper_weight<SPL>(frac_of(pb));
    const float yi = (!CLIP || (i >= R.s_lo && i <= R.s_hi)) ? yw : 0.0f;
    const float g1 = yi * db;                      // to voxel ib + 1
    const float g0 = __fmaf_rn(-yi, db, yi);       // yi (1 - db), to voxel ib
    float x0, x1;
    bool w0, w1;                                     // this lane adds to voxel ib / ib + 1
    combine_lane<RUNS, ASC>(ib, g0, g1, x0, x1, w0, w1);
    float *p = vol + (plane + (Index)ia * sa + (Index)ib);
    const float wa0 = 1.0f - da;
    if (CHECKED) {
        const bool r0 = (unsigned)ia < na, r1 = (unsigned)(ia + 1) < na;   // zero border
        const bool z0 = (unsigned)ib < nb, z1 = (unsigned)(ib + 1) < nb;
        red_add_if(z0 && w0 && r0, p, wa0 * x0);
        red_add_if(z0 && w0 && r1, p + sa, da * x0);
        red_add_if(z1 && w1 && r0, p + 1, wa0 * x1);
        red_add_if(z1 && w1 && r1, p + sa + 1, da * x1);
    } else {
        const bool ok = taps_in_grid(i, ia, ib, R.nm, R.na, R.nb);   // always true but in the debug build
        red_add2_if(ok && w0, p, wa0 * x0, p + sa, da * x0);
        red_add2_if(ok && w1, p + 1, wa0 * x1, p + sa + 1, da * x1);
    }
    pa += (unsigned long long)R.Ga;
    pb += (unsigned long long)R.Gb;
    plane += (Index)R.sm;
}

// One unchecked plane whose row weight and row offset come from the warp's
// row table (entry weight bits, offset).
template <bool SPL, bool RUNS, bool ASC>
__device__ __forceinline__ void combine_row_plane(float yw, unsigned wbits, unsigned off, unsigned long long &pb,
                                                  unsigned long long gb, int sa, float *__restrict__ vol, int i,
                                                  const Ray &R)
{
    // (i: the plane, for the tap check of the debug build)
    const int ib = floor_of(pb);
    const float db = upper_weight<SPL>(frac_of(pb));
    const float g1 = yw * db;
    const float g0 = __fmaf_rn(-yw, db, yw);
    float x0, x1;
    bool w0, w1;
    combine_lane<RUNS, ASC>(ib, g0, g1, x0, x1, w0, w1);
    float *p = vol + (int)(off + (unsigned)ib);
    const float da = __uint_as_float(wbits), wa0 = 1.0f - da;
    const bool ok = row_taps_in_grid(off, i, ib, R);   // always true but in the debug build
    red_add2_if(ok && w0, p, wa0 * x0, p + sa, da * x0);
    red_add2_if(ok && w1, p + 1, wa0 * x1, p + sa + 1, da * x1);
    pb += gb;
}

// Unchecked planes i_lo .. i_hi of a warp on one row (32-bit offsets): the
// row position is stepped once per plane for the whole warp, as in the
// forward's row-table march -- lane k fills the entry of the k-th of the
// next 32 planes, and every lane reads them from shared memory.
template <bool SPL, bool RUNS, bool ASC>
__device__ __forceinline__ void combine_rows(const Ray &R, int i_lo, int i_hi, float yw, unsigned long long &pb,
                                             uint2 *__restrict__ rows, float *__restrict__ vol)
{
    const int lane = threadIdx.x;
    const int sa = (int)R.sa;
    const unsigned long long gb = (unsigned long long)R.Gb;
    unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, i_lo + lane, R.ic);
    const unsigned long long ga32 = (unsigned long long)R.Ga << 5;
    unsigned row = (unsigned)(i_lo + lane) * (unsigned)R.sm;
    const unsigned sm32 = 32u * (unsigned)R.sm;
    for (int w = i_lo; w <= i_hi; w += 32) {
        __syncwarp();                                 // every lane has read the last window
        rows[lane] = make_uint2(__float_as_uint(upper_weight<SPL>(frac_of(pa))),
                                row + (unsigned)floor_of(pa) * (unsigned)sa);
        pa += ga32;
        row += sm32;
        __syncwarp();
        const int n = min(32, i_hi - w + 1);
        int j = 0;
        for (; j + 1 < n; j += 2) {
            const uint4 e = *reinterpret_cast<const uint4 *>(rows + j);
            combine_row_plane<SPL, RUNS, ASC>(yw, e.x, e.y, pb, gb, sa, vol, w + j, R);
            combine_row_plane<SPL, RUNS, ASC>(yw, e.z, e.w, pb, gb, sa, vol, w + j + 1, R);
        }
        if (j < n) {
            const uint2 e = rows[j];
            combine_row_plane<SPL, RUNS, ASC>(yw, e.x, e.y, pb, gb, sa, vol, w + j, R);
        }
    }
}

// The warp's planes I0 .. I1: checked planes before c_end, the planes
// F0 .. F1 that are interior for every lane unchecked (through the row
// table with 32-bit offsets), then checked planes to the end.
template <typename Index, bool SPL, bool CLIP, bool RUNS, bool ASC, bool USE_ROWS>
__device__ __forceinline__ void combine_march(const Ray &R, int I0, int I1, int c_end, int F0, int F1, float yw,
                                              unsigned long long pa, unsigned long long pb, Index plane, Index sa,
                                              unsigned na, unsigned nb, uint2 *__restrict__ rows,
                                              float *__restrict__ vol)
{
    int i = I0;
    for (; i < c_end; ++i)
        combine_plane<Index, SPL, true, CLIP, RUNS, ASC>(R, i, yw, pa, pb, plane, sa, na, nb, vol);
    if (F0 <= F1) {
        const int hi = min(F1, I1);
        if (USE_ROWS && i <= hi) {
            combine_rows<SPL, RUNS, ASC>(R, i, hi, yw, pb, rows, vol);
            i = hi + 1;
            pa = (unsigned long long)pos_at(R.Pa, R.Ga, i, R.ic);
            plane = (Index)i * (Index)R.sm;
        }
        for (; i <= hi; ++i)
            combine_plane<Index, SPL, false, false, RUNS, ASC>(R, i, yw, pa, pb, plane, sa, na, nb, vol);
    }
    for (; i <= I1; ++i)
        combine_plane<Index, SPL, true, CLIP, RUNS, ASC>(R, i, yw, pa, pb, plane, sa, na, nb, vol);
}

template <typename Index, bool SPL, bool CLIP>
__global__ void __launch_bounds__(kMaxThreads) gjp_adjoint_combine_kernel(
    const float *__restrict__ proj, VolParams V, const ViewParams *__restrict__ views,
    int nu, int nv, int n_tv, int n_views, int view_group, float *__restrict__ vol)
{
    int tile, view;
    block_tile_view(n_views, view_group, tile, view);
    const int lane = threadIdx.x;
    const int v_base = (tile % n_tv) * kTileV;
    const int iv = v_base + lane;
    const int iu = (tile / n_tv) * (int)blockDim.y + threadIdx.y;
    if (iu >= nu || v_base >= nv) return;            // the whole warp has no ray
    const unsigned full = 0xffffffffu;

    // lanes past the last detector row trace the ray of their (virtual) row
    // with weight 0
    const bool have = iv < nv;
    const float y = have ? __ldg(proj + ((size_t)view * nv + iv) * nu + iu) : 0.0f;
    ViewParams vp;
    load_view(views, view, vp);
    Ray R;
    setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);
    const float ys = y * R.step;

    const int m0 = __shfl_sync(full, R.m, 0);
    const long long Pa0 = __shfl_sync(full, R.Pa, 0), Ga0 = __shfl_sync(full, R.Ga, 0);
    const bool uniform = __all_sync(full, R.m == m0 && R.Pa == Pa0 && R.Ga == Ga0) && m0 != 2;
    // unchecked planes step the shared row once per warp (32-bit offsets)
    constexpr bool USE_ROWS = GJP_ROWS && std::is_same<Index, int>::value;
    uint2 *rows = row_table(threadIdx.y);
    if (!uniform) {
        if (ys != 0.0f) scatter_ray<Index, SPL>(R, ys, vol);
        return;
    }
    const bool act = ys != 0.0f && R.s_lo <= R.s_hi;
    const int I0 = __reduce_min_sync(full, act ? R.s_lo : 0x7fffffff);
    const int I1 = __reduce_max_sync(full, act ? R.s_hi : -1);
    if (I0 > I1) return;                               // nothing to add (warp-uniform)

    // m in {x, y}: b is z (stride 1); a, ia and da are the same on every
    // lane.  Planes outside a lane's support put its taps outside the grid,
    // where the zero-border checks drop them -- unless the rays are clipped
    // to a field-of-view cylinder (CLIP), where the plane test is explicit.
    const float yw = act ? ys : 0.0f;
    const Index sa = (Index)R.sa, sm = (Index)R.sm;
    const unsigned na = (unsigned)R.na, nb = (unsigned)R.nb;
    unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, I0, R.ic);
    unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, I0, R.ic);
    Index plane = (Index)I0 * sm;

    // Planes F0 .. F1 are interior for every lane of the warp (ghost lanes
    // included: their rays are real rays beyond the detector edge): all
    // four taps of every lane lie in the grid and in the support, so they
    // run without checks; the planes before and after check each tap.
    const int F0 = __reduce_max_sync(full, R.j_lo), F1 = __reduce_min_sync(full, R.j_hi);
    const int c_end = F0 <= F1 ? min(F0, I1 + 1) : I1 + 1;
    // Run form when no three neighbouring lanes can share a voxel: lanes two
    // apart differ by at least one voxel, with one sign, on the first and the
    // last plane (the difference is affine in the plane index, so it then
    // holds in between).
    bool runs_ok = true, asc = true;
    {
        const long long one = 1LL << 32;
        long long d[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const long long p = pos_at(R.Pb, R.Gb, e ? I1 : I0, R.ic);
            d[e] = __shfl_down_sync(full, p, 2) - p;
        }
        if (lane < 30 && !((d[0] >= one && d[1] >= one) || (d[0] <= -one && d[1] <= -one))) runs_ok = false;
        runs_ok = __all_sync(full, runs_ok);
        asc = __shfl_sync(full, d[0] > 0 ? 1 : 0, 0) != 0;   // z order of the lanes (used by the run form)
    }
    if (!runs_ok)
        combine_march<Index, SPL, CLIP, false, true, USE_ROWS>(R, I0, I1, c_end, F0, F1, yw, pa, pb, plane, sa, na, nb,
                                                               rows, vol);
    else if (asc)
        combine_march<Index, SPL, CLIP, true, true, USE_ROWS>(R, I0, I1, c_end, F0, F1, yw, pa, pb, plane, sa, na, nb,
                                                              rows, vol);
    else
        combine_march<Index, SPL, CLIP, true, false, USE_ROWS>(R, I0, I1, c_end, F0, F1, yw, pa, pb, plane, sa, na, nb,
                                                               rows, vol);
}

// ---------------------------------------------------------------------------
// Adjoint, shared-memory slab with TMA bulk reduction.
//
// The transpose of the slab forward: a block of kSlabWarps detector
// columns x 32 rows sweeps its planes kPlanes at a time; each stage's
// contributions are accumulated into a zeroed shared-memory box (the same
// box the forward would load) with shared-memory atomics, and one
// cp.reduce.async.bulk.tensor adds the whole box to the volume in L2.
// This replaces four scattered global reductions per sample by bulk
// sector-wide reductions.  Reductions may not start at a negative
// coordinate, so box origins are clamped to >= 0; taps below index 0 lie
// outside the volume and are skipped, and the TMA unit drops box elements
// beyond the volume.

constexpr int kAdjSlots = 2;

__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap *map, const void *src, int c0, int c1, int c2)
{
    asm volatile(
        "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3, %4}], [%1];"
        ::"l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N> __device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

template <int N> __device__ __forceinline__ void bulk_wait()
{
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct AdjShared {
    int4 hdr[kAdjSlots];            // a0, b0 (clamped to >= 0), box fits, unused
    long long corner[4][4];
    int sweep_lo, sweep_hi, m_first, mixed;
};

template <typename Index, int kBoxC>
__global__ void __launch_bounds__(kSlabWarps * 32, 3) gjp_adjoint_slab_kernel(
    const float *__restrict__ proj, VolParams V, const ViewParams *__restrict__ views, int nu, int nv, int n_tv,
    int n_views, int view_group, const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_y,
    int box_r, float *__restrict__ vol)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int stage_elems = kPlanes * box_r * kBoxC;
    const int stage_bytes = (stage_elems * 4 + 127) & ~127;
    AdjShared &S = *reinterpret_cast<AdjShared *>(smem_raw + kAdjSlots * stage_bytes);
    float *boxes = reinterpret_cast<float *>(smem_raw);
    const int stage_stride = stage_bytes / 4;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    int tile, view;
    block_tile_view(n_views, view_group, tile, view);
    const int v_base = (tile % n_tv) * 32, u_base = (tile / n_tv) * kSlabWarps;
    const int iv = v_base + lane, iu = u_base + warp;
    const bool have_ray = iv < nv && iu < nu;

    if (tid == 0) {
        S.sweep_lo = 0x7fffffff;
        S.sweep_hi = -1;
        S.m_first = -1;
        S.mixed = 0;
    }
    __syncthreads();
    Ray R;
    float ys = 0.0f;
    if (have_ray) {
        ViewParams vp;
        load_view(views, view, vp);
        setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);
        ys = __ldg(proj + ((size_t)view * nv + iv) * nu + iu) * R.step;
        if (R.s_lo <= R.s_hi && ys != 0.0f) {
            atomicMin(&S.sweep_lo, R.s_lo);
            atomicMax(&S.sweep_hi, R.s_hi);
        }
        atomicCAS(&S.m_first, -1, R.m);
    }
    __syncthreads();
    if (have_ray) {
        if (R.m != S.m_first) S.mixed = 1;
        const int u_last = min(kSlabWarps, nu - u_base) - 1, v_last = min(32, nv - v_base) - 1;
        for (int cu = 0; cu < 2; ++cu)
            for (int cv = 0; cv < 2; ++cv)
                if ((cu == 0 ? warp == 0 : warp == u_last) && (cv == 0 ? lane == 0 : lane == v_last)) {
                    long long *c = S.corner[2 * cu + cv];
                    c[0] = R.Pa;
                    c[1] = R.Ga;
                    c[2] = R.Pb;
                    c[3] = R.Gb;
                }
    }
    __syncthreads();
    const int m = S.m_first;
    if (S.mixed || m < 0 || m == 2) {       // global-atomic scatter for the whole tile
        if (have_ray && ys != 0.0f) scatter_ray<Index>(R, ys, vol);
        return;
    }
    const int I0 = S.sweep_lo, I1 = S.sweep_hi;
    const int n_stages = I1 >= I0 ? (I1 - I0) / kPlanes + 1 : 0;
    const int row_stride = m == 0 ? kBoxC : kPlanes * kBoxC;
    const int plane_stride = m == 0 ? box_r * kBoxC : kBoxC;
    const int nm = V.n[m];
    const int ic = (nm - 1) >> 1;
    const unsigned na = have_ray ? (unsigned)R.na : 0u, nb = have_ray ? (unsigned)R.nb : 0u;
    const Index sa = have_ray ? (Index)R.sa : 0, sb = have_ray ? (Index)R.sb : 0, sm = have_ray ? (Index)R.sm : 0;
    unsigned long long pa = 0, pb = 0, ga = 0, gb = 0;
    int s_lo = 1, s_hi = 0;
    if (have_ray && ys != 0.0f) {
        pa = (unsigned long long)pos_at(R.Pa, R.Ga, I0, R.ic);
        pb = (unsigned long long)pos_at(R.Pb, R.Gb, I0, R.ic);
        ga = (unsigned long long)R.Ga;
        gb = (unsigned long long)R.Gb;
        s_lo = R.s_lo;
        s_hi = R.s_hi;
    }
    // corner tracked by this lane of warp 0 (stage box from the corners at
    // the stage's first and last plane, as in the forward)
    const long long *cr = S.corner[lane & 3];
    const long long cPa = cr[0], cGa = cr[1], cPb = cr[2], cGb = cr[3];
    const int cend = (lane >> 2) & 1;

    for (int st = 0; st < n_stages; ++st) {
        const int slot = st & (kAdjSlots - 1);
        float *box = boxes + slot * stage_stride;
        const int i0 = I0 + st * kPlanes;
        if (warp == 0) {
            const int i = cend ? min(i0 + kPlanes - 1, I1) : i0;
            const int fa = floor_of((unsigned long long)pos_at(cPa, cGa, i, ic));
            const int fb = floor_of((unsigned long long)pos_at(cPb, cGb, i, ic));
            const int amin = __reduce_min_sync(0xffffffffu, fa), amax = __reduce_max_sync(0xffffffffu, fa);
            const int bmin = __reduce_min_sync(0xffffffffu, fb), bmax = __reduce_max_sync(0xffffffffu, fb);
            if (lane == 0) {
                const int a0 = amin - 1;
                const int b0 = (bmin - 1) & ~3;
                const bool fits = (amax + 3 - a0 <= box_r) && (bmax + 3 - b0 <= kBoxC);
                S.hdr[slot] = make_int4(max(a0, 0), max(b0, 0), fits ? 1 : 0, 0);
                // the reduction issued kAdjSlots stages ago from this slot must
                // have finished reading it before it is zeroed again
                bulk_wait_read<kAdjSlots - 1>();
            }
        }
        __syncthreads();                                    // header visible, slot free
        const int4 h = S.hdr[slot];
        if (h.z) {
            float4 *b4 = reinterpret_cast<float4 *>(box);
            for (int k = tid; k < stage_elems / 4; k += kSlabWarps * 32) b4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();                                    // box zeroed
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const int i = i0 + p;
            if (i >= s_lo && i <= s_hi) {
                const float da = frac_of(pa), db = frac_of(pb);
                const int ia = floor_of(pa), ib = floor_of(pb);
                const float w0 = (1.0f - da) * ys, w1 = da * ys;
                const float w00 = w0 * (1.0f - db), w01 = w0 * db, w10 = w1 * (1.0f - db), w11 = w1 * db;
                if (h.z) {
                    const int r = ia - h.x, c = ib - h.y;   // r, c >= -1; -1 only outside the volume
                    float *q = box + (r * row_stride + c + p * plane_stride);
                    const bool r0 = r >= 0, c0 = c >= 0;
                    if (r0 && c0) atomicAdd(q, w00);
                    if (r0) atomicAdd(q + 1, w01);
                    if (c0) atomicAdd(q + row_stride, w10);
                    atomicAdd(q + row_stride + 1, w11);
                } else {
                    const bool a0 = (unsigned)ia < na, a1 = (unsigned)(ia + 1) < na;
                    const bool b0 = (unsigned)ib < nb, b1 = (unsigned)(ib + 1) < nb;
                    float *q = vol + ((Index)i * sm + (Index)ia * sa + (Index)ib * sb);
                    if (a0 && b0) atomicAdd(q, w00);
                    if (a0 && b1) atomicAdd(q + sb, w01);
                    if (a1 && b0) atomicAdd(q + sa, w10);
                    if (a1 && b1) atomicAdd(q + sa + sb, w11);
                }
            }
            pa += ga;
            pb += gb;
        }
        fence_proxy_async_smem();                           // box writes -> async proxy
        __syncthreads();                                    // box complete
        if (tid == 0 && h.z) {
            if (m == 0) tma_reduce_add_3d(&map_x, box, h.y, h.x, i0);     // planes x = i0 ..
            else tma_reduce_add_3d(&map_y, box, h.y, i0, h.x);            // planes y = i0 ..
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait<0>();
}

// Marks every voxel that receives a non-zero interpolation weight from a
// ray of one view (the view's compulsory volume traffic).
template <typename Index>
__global__ void __launch_bounds__(kMaxThreads) gjp_footprint_kernel(
    VolParams V, const ViewParams *__restrict__ views, int view, int nu, int nv, int n_tv,
    unsigned char *__restrict__ marks)
{
    const int tile = blockIdx.x;
    const int iv = (tile % n_tv) * kTileV + threadIdx.x;
    const int iu = (tile / n_tv) * (int)blockDim.y + threadIdx.y;
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

VolParams make_vol(const int64_t n[3], const double h[3], double fov)
{
    VolParams V;
    V.fov_r2 = fov > 0.0 ? (float)(fov * fov) : 0.0f;
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

size_t elem_size(gjp_dtype t) { return t == GJP_F32 ? 4 : 2; }

void fit_carveout(const void *func, int threads, size_t dyn_smem)
{
    int dev = 0, per_sm = 0, smem_sm = 0, reserved = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, dyn_smem) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, func) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        per_sm < 1 || smem_sm < 1) {
        cudaGetLastError();
        return;
    }
    const size_t need = (size_t)per_sm * (fa.sharedSizeBytes + dyn_smem + (size_t)reserved);
    const int pct = (int)std::min<size_t>(100, (need * 100 + (size_t)smem_sm - 1) / (size_t)smem_sm);
    int after = 0;
    if (cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&after, func, threads, dyn_smem) != cudaSuccess ||
        after < per_sm)
        cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, -1);
    cudaGetLastError();
}

// cuTensorMapEncodeTiled, fetched once through the runtime (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Host (FP64) sizing of the slab boxes: for sample tiles of every view (the
// 3 x 3 grid of tiles at the panel's corners, edge midpoints and centre,
// where footprints are largest), the per-plane box the kernel's producer
// computes from the tile's corner rays, over the planes some corner ray
// supports.  Planes whose box still exceeds the chosen size fall back to
// the gather path inside the kernel, so this only has to be typical.
struct BoxSize {
    int rows, cols4, cols8;   // cols for a 4- and an 8-element TMA x granularity
};

BoxSize slab_box_size(const gjp_geometry &g, const int64_t n[3], const double h[3], const double o[3])
{
    BoxSize bs{0, 0, 0};
    const int us[3] = {0, std::max(0, g.nu / 2 - kSlabWarps / 2), std::max(0, g.nu - kSlabWarps)};
    const int vs[3] = {0, std::max(0, g.nv / 2 - 16), std::max(0, g.nv - 32)};
    for (int k = 0; k < g.n_views; ++k) {
        double s[3];
        for (int a = 0; a < 3; ++a) s[a] = (g.src[3 * k + a] - o[a]) / h[a];
        for (int tu = 0; tu < 3; ++tu)
            for (int tv = 0; tv < 3; ++tv) {
                const int u0 = us[tu], v0 = vs[tv];
                const int u1 = std::min(g.nu - 1, u0 + kSlabWarps - 1), v1 = std::min(g.nv - 1, v0 + 31);
                const int cu[4] = {u0, u0, u1, u1}, cv[4] = {v0, v1, v0, v1};
                double r[4][3];
                int m = -1;
                bool mixed = false;
                for (int c = 0; c < 4; ++c) {
                    for (int a = 0; a < 3; ++a) {
                        const double d = g.org[3 * k + a] + cu[c] * g.du[3 * k + a] + cv[c] * g.dv[3 * k + a];
                        r[c][a] = (d - o[a]) / h[a] - s[a];
                    }
                    int mc = 0;
                    for (int a = 1; a < 3; ++a)
                        if (std::fabs(r[c][a]) > std::fabs(r[c][mc])) mc = a;
                    if (m >= 0 && mc != m) mixed = true;
                    m = mc;
                }
                if (mixed || m == 2) continue;
                const int a = m == 0 ? 1 : 0, b = 2;
                for (int64_t i = 0; i < n[m]; ++i) {
                    double amin = 1e300, amax = -1e300, bmin = 1e300, bmax = -1e300;
                    bool sup = false;
                    for (int c = 0; c < 4; ++c)
                        for (int e = 0; e < 2; ++e) {   // first and last plane of a stage
                            const double ip = e ? (double)std::min<int64_t>(i + kPlanes - 1, n[m] - 1) : (double)i;
                            const double t = (ip - s[m]) / r[c][m];
                            const double pa = s[a] + t * r[c][a], pb = s[b] + t * r[c][b];
                            amin = std::min(amin, pa);
                            amax = std::max(amax, pa);
                            bmin = std::min(bmin, pb);
                            bmax = std::max(bmax, pb);
                            if (!e && pa > -1.0 && pa < (double)n[a] && pb > -1.0 && pb < (double)n[b]) sup = true;
                        }
                    if (!sup) continue;
                    const int a0 = (int)std::floor(amin) - 1;
                    const int fb = (int)std::floor(bmin) - 1;
                    const int b04 = fb - ((fb % 4) + 4) % 4, b08 = fb - ((fb % 8) + 8) % 8;
                    const int bmx = (int)std::floor(bmax);
                    bs.rows = std::max(bs.rows, (int)std::floor(amax) + 3 - a0);
                    bs.cols4 = std::max(bs.cols4, bmx + 3 - b04);
                    bs.cols8 = std::max(bs.cols8, bmx + 3 - b08);
                }
            }
    }
    return bs;
}

struct SlabPlan {
    bool ok;
    int rows, cols;
};

SlabPlan slab_plan(const BoxSize &bs, const void *vol, gjp_dtype dt, const int64_t n[3])
{
    SlabPlan p{false, 0, 0};
    const size_t es = elem_size(dt);
    if (((uintptr_t)vol % 16) != 0 || ((size_t)n[2] * es) % 16 != 0) return p;
    if (!tensor_map_encoder() || bs.rows <= 0) return p;
    const int cols_need = es == 4 ? bs.cols4 : bs.cols8;
    if (bs.rows > kBoxRMax || cols_need > 72) return p;   // too many planes would fall back
    p.rows = std::max(4, bs.rows);
    p.cols = cols_need <= (es == 4 ? 48 : 56) ? (es == 4 ? 48 : 56) : 64;
    p.ok = true;
    return p;
}

bool encode_maps(const void *vol, gjp_dtype dt, const int64_t n[3], int rows, int cols, CUtensorMap *mx,
                 CUtensorMap *my)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const size_t es = elem_size(dt);
    const CUtensorMapDataType t = dt == GJP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                  : dt == GJP_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)n[2], (cuuint64_t)n[1], (cuuint64_t)n[0]};
    const cuuint64_t strides[2] = {(cuuint64_t)(n[2] * es), (cuuint64_t)(n[1] * n[2] * es)};
    const cuuint32_t bx[3] = {(cuuint32_t)cols, (cuuint32_t)rows, (cuuint32_t)kPlanes};   // planes x = i..: rows along y
    const cuuint32_t by[3] = {(cuuint32_t)cols, (cuuint32_t)kPlanes, (cuuint32_t)rows};   // planes y = i..: rows along x
    const cuuint32_t es1[3] = {1, 1, 1};
    void *base = const_cast<void *>(vol);
    if (enc(mx, t, 3, base, dims, strides, bx, es1, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (enc(my, t, 3, base, dims, strides, by, es1, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    return true;
}

template <typename T, typename Index, int C>
cudaError_t launch_slab(const T *vol, const VolParams &V, const ViewParams *table, const gjp_geometry &g,
                        const CUtensorMap &mx, const CUtensorMap &my, int rows, float *proj, cudaStream_t s)
{
    const int n_tv = (g.nv + 31) / 32;
    const int n_tu = (g.nu + kSlabWarps - 1) / kSlabWarps;
    const dim3 grid((unsigned)(n_tv * n_tu), (unsigned)g.n_views);
    const int stage_bytes = (kPlanes * rows * C * (int)sizeof(T) + 127) & ~127;
    const size_t smem = (size_t)kStages * stage_bytes + sizeof(SlabShared);
    auto kern = gjp_forward_slab_kernel<T, Index, C>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, kSlabThreads, smem, s>>>(vol, V, table, g.nu, g.nv, n_tv, g.n_views, launch_view_group(g, V.n), mx, my, rows,
                                          proj);
    return cudaGetLastError();
}

template <typename T, typename Index>
cudaError_t launch_slab_cols(const T *vol, const VolParams &V, const ViewParams *table, const gjp_geometry &g,
                             const CUtensorMap &mx, const CUtensorMap &my, const SlabPlan &p, float *proj,
                             cudaStream_t s)
{
    if (p.cols == 48) return launch_slab<T, Index, 48>(vol, V, table, g, mx, my, p.rows, proj, s);
    if (p.cols == 56) return launch_slab<T, Index, 56>(vol, V, table, g, mx, my, p.rows, proj, s);
    return launch_slab<T, Index, 64>(vol, V, table, g, mx, my, p.rows, proj, s);
}

bool encode_prefetch_map(const void *vol, gjp_dtype dt, const int64_t n[3], CUtensorMap *map)
{
    auto enc = tensor_map_encoder();
    const size_t es = elem_size(dt);
    if (!enc || ((uintptr_t)vol % 16) != 0 || ((size_t)n[2] * es) % 16 != 0) return false;
    const CUtensorMapDataType t = dt == GJP_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                  : dt == GJP_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)n[2], (cuuint64_t)n[1], (cuuint64_t)n[0]};
    const cuuint64_t strides[2] = {(cuuint64_t)(n[2] * es), (cuuint64_t)(n[1] * n[2] * es)};
    // the same box serves planes x = i (rows along y) and planes y = i (rows along x)
    static_assert(kPfRows == kPlanes, "prefetch box is square in rows and planes");
    const cuuint32_t box[3] = {(cuuint32_t)(es == 4 ? 48 : 64), (cuuint32_t)kPfRows, (cuuint32_t)kPlanes};
    const cuuint32_t es1[3] = {1, 1, 1};
    return enc(map, t, 3, const_cast<void *>(vol), dims, strides, box, es1, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
cudaError_t launch_gather_pf(const T *vol, gjp_dtype dt, const int64_t n[3], const VolParams &V,
                             const ViewParams *table, const gjp_geometry &g, bool i32, float *proj, cudaStream_t s,
                             bool &launched)
{
    launched = false;
    CUtensorMap map;
    if (!encode_prefetch_map(vol, dt, n, &map)) return cudaSuccess;
    const int n_tv = (g.nv + kTileV - 1) / kTileV;
    const int n_tu = (g.nu + g.tile_u - 1) / g.tile_u;
    const dim3 grid((unsigned)(n_tv * n_tu), (unsigned)g.n_views);
    const dim3 block(kTileV, g.tile_u);
    if (i32)
        gjp_forward_pf_kernel<T, int><<<grid, block, 0, s>>>(vol, V, table, g.nu, g.nv, n_tv, g.n_views, launch_view_group(g, V.n),
                                                             map, proj);
    else
        gjp_forward_pf_kernel<T, long long><<<grid, block, 0, s>>>(vol, V, table, g.nu, g.nv, n_tv, g.n_views,
                                                                   launch_view_group(g, V.n), map, proj);
    launched = true;
    return cudaGetLastError();
}

// pairs: the z-paired copy of vol for the row-table march (32-bit offsets
// only), or null to read the taps from vol.
template <typename T>
cudaError_t launch_gather_shaped(const T *vol, const VolParams &V, const ViewParams *table, const GatherShape &sh,
                                 bool i32, float *proj, cudaStream_t s,
                                 const typename PairOf<T>::type *pairs = nullptr)
{
    const int n_tv = (sh.nv + kTileV - 1) / kTileV;
    const int n_tu = (sh.nu + sh.tile_u - 1) / sh.tile_u;
    const dim3 grid((unsigned)(n_tv * n_tu), (unsigned)sh.n_views);
    const dim3 block(kTileV, sh.tile_u);
    const bool spl = sh.spl;
    const int nu = sh.nu, nv = sh.nv, nvw = sh.n_views, vgp = sh.view_group;
    const size_t rows = (size_t)sh.tile_u * 32 * sizeof(uint2);   // row tables (32-bit offsets only)
#define GJP_LAUNCH_FWD(I, S, P, SMEM)                                                                              \
    gjp_forward_kernel<T, I, S, P><<<grid, block, SMEM, s>>>(vol, V, table, nu, nv, n_tv, nvw, vgp, proj, pairs)
    if (i32 && pairs) {
        if (spl) GJP_LAUNCH_FWD(int, true, true, rows);
        else GJP_LAUNCH_FWD(int, false, true, rows);
    } else if (i32) {
        if (spl) GJP_LAUNCH_FWD(int, true, false, rows);
        else GJP_LAUNCH_FWD(int, false, false, rows);
    } else {
        if (spl) GJP_LAUNCH_FWD(long long, true, false, 0);
        else GJP_LAUNCH_FWD(long long, false, false, 0);
    }
#undef GJP_LAUNCH_FWD
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather(const T *vol, const VolParams &V, const ViewParams *table, const gjp_geometry &g,
                          bool i32, float *proj, cudaStream_t s, const typename PairOf<T>::type *pairs = nullptr)
{
    const GatherShape sh{g.nu, g.nv, g.n_views, g.tile_u, launch_view_group(g, V.n), g.weight == GJP_WEIGHT_SPL};
    return launch_gather_shaped<T>(vol, V, table, sh, i32, proj, s, pairs);
}

// Writes the z-paired copy of vol (n[0] n[1] lines of n[2] voxels) to out.
// 16-bit volumes whose lines are whole 8-byte words take the 4-voxel form.
template <typename T>
cudaError_t launch_zpairs(const T *vol, const int64_t n[3], typename PairOf<T>::type *out, cudaStream_t s)
{
    const long long lines = (long long)n[0] * n[1];
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = std::min<long long>(lines, (long long)std::max(sms, 1) * 8);
    if constexpr (!std::is_same<T, float>::value) {
        if (n[2] % 4 == 0 && reinterpret_cast<uintptr_t>(vol) % 8 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0) {
            const int quads = (int)(n[2] / 4);
            const int threads = quads >= 128 ? 128 : 32 * ((quads + 31) / 32);
            gjp_zpairs16x4_kernel<<<(unsigned)blocks, threads, 0, s>>>(
                reinterpret_cast<const unsigned short *>(vol), lines, (int)n[2], reinterpret_cast<uint4 *>(out));
            return cudaGetLastError();
        }
    }
    const int threads = n[2] >= 256 ? 256 : 128;
    gjp_zpairs_kernel<T><<<(unsigned)blocks, threads, 0, s>>>(vol, lines, (int)n[2], out);
    return cudaGetLastError();
}

cudaError_t forward_gather_shaped(const void *vol, gjp_dtype dt, const VolParams &V, const ViewParams *table,
                                  const GatherShape &sh, bool i32, float *proj, const void *pairs, cudaStream_t s)
{
    switch (dt) {
    case GJP_F32:
        return launch_gather_shaped<float>(static_cast<const float *>(vol), V, table, sh, i32, proj, s);
    case GJP_BF16:
        return launch_gather_shaped<__nv_bfloat16>(static_cast<const __nv_bfloat16 *>(vol), V, table, sh, i32, proj, s,
                                                   static_cast<const unsigned *>(pairs));
    default:
        return launch_gather_shaped<__half>(static_cast<const __half *>(vol), V, table, sh, i32, proj, s,
                                            static_cast<const unsigned *>(pairs));
    }
}

cudaError_t write_zpairs16(const void *vol, gjp_dtype dt, const int64_t n[3], void *out, cudaStream_t s)
{
    if (dt == GJP_BF16)
        return launch_zpairs<__nv_bfloat16>(static_cast<const __nv_bfloat16 *>(vol), n, static_cast<unsigned *>(out), s);
    return launch_zpairs<__half>(static_cast<const __half *>(vol), n, static_cast<unsigned *>(out), s);
}

template <typename T>
gjp_status forward_typed(const void *d_volume, gjp_dtype dt, const int64_t n[3], const double h[3],
                         const double o[3], const gjp_geometry &g, gjp_cache_entry &entry, float *proj,
                         int path, cudaStream_t s)
{
    const VolParams V = make_vol(n, h, g.fov);
    const bool i32 = fits_int32(n);
    const T *vol = static_cast<const T *>(d_volume);
    const ViewParams *table = entry.d_table;
    if (path == GJP_PATH_TEXTURE || path == GJP_PATH_HWLIN)
        return forward_texture(d_volume, dt, n, V, g, entry, proj, path, s);
    if ((path == GJP_PATH_PREFETCH || path == GJP_PATH_SLAB) && g.weight != GJP_WEIGHT_LIN)
        return GJP_ERR_UNSUPPORTED;   // those families implement w_lin only
    if (path == GJP_PATH_PREFETCH) {
        bool launched = false;
        const cudaError_t e = launch_gather_pf<T>(vol, dt, n, V, table, g, i32, proj, s, launched);
        if (!launched) return GJP_ERR_UNSUPPORTED;
        return e == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
    }
    // measured on the 512^3 / 512^2 / 360-view workload the gather family is
    // the fastest, so AUTO takes it; SLAB and PREFETCH run only on request
    if (path == GJP_PATH_SLAB) {
        BoxSize bs;
        {
            std::lock_guard<std::mutex> lock(const_cast<gjp_geometry &>(g).mu);
            if (entry.box_rows == 0) {
                const BoxSize b = slab_box_size(g, n, h, o);
                entry.box_rows = std::max(b.rows, 1);
                entry.box_cols4 = b.cols4;
                entry.box_cols8 = b.cols8;
            }
            bs = BoxSize{entry.box_rows, entry.box_cols4, entry.box_cols8};
        }
        const SlabPlan p = slab_plan(bs, d_volume, dt, n);
        CUtensorMap mx, my;
        if (p.ok && encode_maps(d_volume, dt, n, p.rows, p.cols, &mx, &my)) {
            const cudaError_t e = i32 ? launch_slab_cols<T, int>(vol, V, table, g, mx, my, p, proj, s)
                                      : launch_slab_cols<T, long long>(vol, V, table, g, mx, my, p, proj, s);
            return e == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
        }
        if (path == GJP_PATH_SLAB) return GJP_ERR_UNSUPPORTED;
    }
    // The z-paired copy: on request (PAIRS), and taken by AUTO for 16-bit
    // storage when pairs_pay(), the offsets fit 32 bits and the copy can be
    // allocated (otherwise AUTO reads the volume directly).  Its results are
    // bitwise those of GATHER.  Measured on the 512^3 / 360-view workload it
    // makes the 16-bit forward 11% faster (copy included) and the float32
    // one 35% slower (8-byte words: twice the footprint in L1 and L2).
    constexpr bool kPairsAuto = !std::is_same<T, float>::value;
    if (path == GJP_PATH_PAIRS || (path == GJP_PATH_AUTO && kPairsAuto && i32 && pairs_pay(g.n_views, n))) {
        if (!i32) return GJP_ERR_UNSUPPORTED;
        using P = typename PairOf<T>::type;
        void *ws = nullptr;
        const gjp_status st = pairs_alloc((size_t)(n[0] * n[1] * n[2]) * sizeof(P), s, &ws);
        if (st == GJP_OK) {
            P *pairs = static_cast<P *>(ws);
            cudaError_t e = launch_zpairs<T>(vol, n, pairs, s);
            if (e == cudaSuccess) e = launch_gather<T>(vol, V, table, g, i32, proj, s, pairs);
            const cudaError_t f = cudaFreeAsync(pairs, s);
            return e == cudaSuccess && f == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
        }
        if (path == GJP_PATH_PAIRS || st == GJP_ERR_CUDA) return st;
    }
    return launch_gather<T>(vol, V, table, g, i32, proj, s) == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

template <typename Index, int C>
cudaError_t launch_adjoint_slab(const float *proj, const VolParams &V, const ViewParams *table,
                                const gjp_geometry &g, const CUtensorMap &mx, const CUtensorMap &my, int rows,
                                float *vol, cudaStream_t s)
{
    const int n_tv = (g.nv + 31) / 32;
    const int n_tu = (g.nu + kSlabWarps - 1) / kSlabWarps;
    const dim3 grid((unsigned)(n_tv * n_tu), (unsigned)g.n_views);
    const int stage_bytes = (kPlanes * rows * C * 4 + 127) & ~127;
    const size_t smem = (size_t)kAdjSlots * stage_bytes + sizeof(AdjShared);
    auto kern = gjp_adjoint_slab_kernel<Index, C>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, kSlabWarps * 32, smem, s>>>(proj, V, table, g.nu, g.nv, n_tv, g.n_views, launch_view_group(g, V.n), mx, my,
                                             rows, vol);
    return cudaGetLastError();
}

// Slab adjoint when its conditions hold; returns false (nothing launched) otherwise.
bool try_adjoint_slab(const float *proj, const int64_t n[3], const double h[3], const double o[3],
                      const gjp_geometry &g, gjp_cache_entry &entry, float *vol, cudaStream_t s, cudaError_t &err)
{
    BoxSize bs;
    {
        std::lock_guard<std::mutex> lock(const_cast<gjp_geometry &>(g).mu);
        if (entry.box_rows == 0) {
            const BoxSize b = slab_box_size(g, n, h, o);
            entry.box_rows = std::max(b.rows, 1);
            entry.box_cols4 = b.cols4;
            entry.box_cols8 = b.cols8;
        }
        bs = BoxSize{entry.box_rows, entry.box_cols4, entry.box_cols8};
    }
    const SlabPlan p = slab_plan(bs, vol, GJP_F32, n);
    CUtensorMap mx, my;
    if (!p.ok || !encode_maps(vol, GJP_F32, n, p.rows, p.cols, &mx, &my)) return false;
    const VolParams V = make_vol(n, h, g.fov);
    const bool i32 = fits_int32(n);
    if (p.cols == 48)
        err = i32 ? launch_adjoint_slab<int, 48>(proj, V, entry.d_table, g, mx, my, p.rows, vol, s)
                  : launch_adjoint_slab<long long, 48>(proj, V, entry.d_table, g, mx, my, p.rows, vol, s);
    else
        err = i32 ? launch_adjoint_slab<int, 64>(proj, V, entry.d_table, g, mx, my, p.rows, vol, s)
                  : launch_adjoint_slab<long long, 64>(proj, V, entry.d_table, g, mx, my, p.rows, vol, s);
    return true;
}

// ---------------------------------------------------------------------------
// Allocation-free forward projection.
//
// gjp_forward builds its per-view table in device memory it allocates with
// cudaMalloc on first use.  Some callers cannot allow that: code that runs
// after a fixed device-memory budget has been handed out (a framework that
// owns the whole device pool, a real-time reconstruction loop that may not
// allocate once acquisition starts), or a plug-in that must not touch the
// allocator of its host application.  gjp_forward_noalloc serves them: its
// table lives in the fixed array below, which the CUDA runtime places in
// device memory when it loads this library onto a GPU and keeps there until
// the process exits.

constexpr int kNoAllocMaxViews = GJP_NOALLOC_MAX_VIEWS;
static __device__ __align__(256) unsigned char g_noalloc_table[kNoAllocMaxViews * sizeof(ViewParams)];

// The table reaches the array as the by-value parameters of a small copy
// kernel, a chunk of views per launch (9 KiB of parameters; the launch
// takes its own copy of them, so no host buffer has to outlive the call).
constexpr int kNoAllocChunk = 64;
struct NoAllocChunk {
    ViewParams v[kNoAllocChunk];
};

__global__ void gjp_noalloc_fill_kernel(const __grid_constant__ NoAllocChunk c, int k0, int cnt)
{
    const unsigned *src = reinterpret_cast<const unsigned *>(c.v);
    unsigned *dst = reinterpret_cast<unsigned *>(reinterpret_cast<ViewParams *>(g_noalloc_table) + k0);
    const int words = cnt * (int)(sizeof(ViewParams) / sizeof(unsigned));
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

// Host side: device address of g_noalloc_table for each device, looked up
// once per device (with that device current) by the first call there.
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices];

gjp_status noalloc_table_address(int dev, ViewParams **out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return GJP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_table) != cudaSuccess || !p) {
            cudaGetLastError();
            return GJP_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<ViewParams *>(g_noalloc_ptr[dev]);
    return GJP_OK;
}

}  // namespace gjp_detail

using namespace gjp_detail;

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
        g->view_step = central_ray_step(*g);
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
            cudaSetDevice(e.device);
            if (e.d_table) cudaFree(e.d_table);
            free_texture_cache(e);
        }
        if (have_dev) cudaSetDevice(cur);
    }
    delete g;
}

gjp_status gjp_geometry_set_weight(gjp_geometry *g, gjp_weight w)
{
    if (!g || (w != GJP_WEIGHT_LIN && w != GJP_WEIGHT_SPL)) return GJP_ERR_INVALID_ARG;
    g->weight = w;
    return GJP_OK;
}

gjp_status gjp_geometry_set_launch(gjp_geometry *g, int tile_u, int view_group)
{
    if (!g || (tile_u != 1 && tile_u != 2 && tile_u != 4 && tile_u != 8) || view_group < 1 || view_group > 64)
        return GJP_ERR_INVALID_ARG;
    g->tile_u = tile_u;
    g->view_group = view_group;
    g->launch_set = true;
    return GJP_OK;
}

gjp_status gjp_geometry_set_fov(gjp_geometry *g, double radius)
{
    if (!g || !std::isfinite(radius) || radius < 0.0) return GJP_ERR_INVALID_ARG;
    g->fov = radius;
    return GJP_OK;
}

gjp_status gjp_geometry_get_launch(const gjp_geometry *g, int *tile_u, int *view_group)
{
    if (!g) return GJP_ERR_INVALID_ARG;
    if (tile_u) *tile_u = g->tile_u;
    if (view_group) *view_group = g->view_group;
    return GJP_OK;
}

gjp_status gjp_geometry_info(const gjp_geometry *g, int *n_views, int *nu, int *nv)
{
    if (!g) return GJP_ERR_INVALID_ARG;
    if (n_views) *n_views = g->n_views;
    if (nu) *nu = g->nu;
    if (nv) *nv = g->nv;
    return GJP_OK;
}

gjp_status gjp_forward_ex(const void *d_volume, gjp_dtype dtype, int64_t nx, int64_t ny, int64_t nz,
                          const double voxel_size[3], const double volume_origin[3], const gjp_geometry *g,
                          float *d_proj, gjp_path path, void *stream)
{
    NvtxRange nvtx_range("gjp_forward");
    if (!d_volume || !g || !d_proj) return GJP_ERR_INVALID_ARG;
    if (dtype != GJP_F32 && dtype != GJP_BF16 && dtype != GJP_F16) return GJP_ERR_INVALID_ARG;
    if (path != GJP_PATH_AUTO && path != GJP_PATH_GATHER && path != GJP_PATH_SLAB && path != GJP_PATH_PREFETCH &&
        path != GJP_PATH_TEXTURE && path != GJP_PATH_HWLIN && path != GJP_PATH_PAIRS)
        return GJP_ERR_INVALID_ARG;
    int64_t n[3];
    double h[3], o[3];
    gjp_status st = check_grid(nx, ny, nz, voxel_size, volume_origin, n, h, o);
    if (st != GJP_OK) return st;
    if ((st = check_sources(g, n, h, o)) != GJP_OK) return st;
    if (g->n_views > 65535) return GJP_ERR_UNSUPPORTED;
    gjp_cache_entry *entry = nullptr;
    if ((st = get_table(g, n, h, o, &entry)) != GJP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    switch (dtype) {
    case GJP_F32: return forward_typed<float>(d_volume, dtype, n, h, o, *g, *entry, d_proj, path, s);
    case GJP_BF16: return forward_typed<__nv_bfloat16>(d_volume, dtype, n, h, o, *g, *entry, d_proj, path, s);
    case GJP_F16: return forward_typed<__half>(d_volume, dtype, n, h, o, *g, *entry, d_proj, path, s);
    }
    return GJP_ERR_INVALID_ARG;
}

gjp_status gjp_forward(const void *d_volume, gjp_dtype dtype, int64_t nx, int64_t ny, int64_t nz,
                       const double voxel_size[3], const double volume_origin[3], const gjp_geometry *g,
                       float *d_proj, void *stream)
{
    return gjp_forward_ex(d_volume, dtype, nx, ny, nz, voxel_size, volume_origin, g, d_proj, GJP_PATH_AUTO,
                          stream);
}

gjp_status gjp_forward_noalloc(const void *d_volume, gjp_dtype dtype, int64_t nx, int64_t ny, int64_t nz,
                               const double voxel_size[3], const double volume_origin[3], const gjp_geometry *g,
                               float *d_proj, void *stream)
{
    NvtxRange nvtx_range("gjp_forward_noalloc");
    if (!d_volume || !g || !d_proj) return GJP_ERR_INVALID_ARG;
    if (dtype != GJP_F32 && dtype != GJP_BF16 && dtype != GJP_F16) return GJP_ERR_INVALID_ARG;
    int64_t n[3];
    double h[3], o[3];
    gjp_status st = check_grid(nx, ny, nz, voxel_size, volume_origin, n, h, o);
    if (st != GJP_OK) return st;
    if (g->n_views > kNoAllocMaxViews) return GJP_ERR_UNSUPPORTED;
    if ((st = check_sources(g, n, h, o)) != GJP_OK) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GJP_ERR_CUDA;
    ViewParams *d_table = nullptr;
    if ((st = noalloc_table_address(dev, &d_table)) != GJP_OK) return st;

    // the per-view table is formed on the host, a chunk of views at a time,
    // and written into the fixed device array by a copy kernel on the
    // caller's stream ahead of the kernel that reads it
    cudaStream_t s = (cudaStream_t)stream;
    NoAllocChunk chunk;
    for (int k0 = 0; k0 < g->n_views; k0 += kNoAllocChunk) {
        const int cnt = std::min(kNoAllocChunk, g->n_views - k0);
        for (int j = 0; j < cnt; ++j) make_view_params(*g, k0 + j, n, h, o, chunk.v[j]);
        gjp_noalloc_fill_kernel<<<1, 256, 0, s>>>(chunk, k0, cnt);
        if (cudaGetLastError() != cudaSuccess) return GJP_ERR_CUDA;
    }
    const VolParams V = make_vol(n, h, g->fov);
    const bool i32 = fits_int32(n);
    cudaError_t e = cudaSuccess;
    switch (dtype) {
    case GJP_F32: e = launch_gather<float>((const float *)d_volume, V, d_table, *g, i32, d_proj, s); break;
    case GJP_BF16:
        e = launch_gather<__nv_bfloat16>((const __nv_bfloat16 *)d_volume, V, d_table, *g, i32, d_proj, s);
        break;
    case GJP_F16: e = launch_gather<__half>((const __half *)d_volume, V, d_table, *g, i32, d_proj, s); break;
    }
    return e == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

gjp_status gjp_selftest_wait_timeout(void *stream)
{
    gjp_wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>();
    return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

gjp_status gjp_debug_fail_allocations(int n)
{
    if (n < 0) return GJP_ERR_INVALID_ARG;
    g_fail_allocations.store(n);
    return GJP_OK;
}

gjp_status gjp_trim_workspace(void)
{
    std::lock_guard<std::mutex> lock(g_pairs_mu);
    for (const auto &p : g_pairs_pools)
        if (cudaMemPoolTrimTo(p.second, 0) != cudaSuccess) return GJP_ERR_CUDA;
    return GJP_OK;
}

gjp_status gjp_selftest_tap_check(void *stream)
{
    if (!GJP_CHECK_TAPS) return GJP_ERR_UNSUPPORTED;
    gjp_tap_check_selftest_kernel<<<1, 1, 0, (cudaStream_t)stream>>>();
    return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

gjp_status gjp_stream_status(void *stream)
{
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GJP_ERR_CUDA;
    if (GJP_CHECK_TAPS) {
        const unsigned taps = take_tap_faults() | batch_tap_faults() | texture_tap_faults();
        if (taps) return GJP_ERR_INTERNAL;
    }
    unsigned flag = 0;
    if (cudaMemcpyFromSymbol(&flag, g_gjp_status, sizeof flag) != cudaSuccess) return GJP_ERR_CUDA;
    if (flag) {
        const unsigned zero = 0;
        if (cudaMemcpyToSymbol(g_gjp_status, &zero, sizeof zero) != cudaSuccess) return GJP_ERR_CUDA;
        return GJP_ERR_TIMEOUT;
    }
    return GJP_OK;
}

gjp_status gjp_adjoint_ex(const float *d_proj, const gjp_geometry *g, int64_t nx, int64_t ny, int64_t nz,
                          const double voxel_size[3], const double volume_origin[3], float *d_volume,
                          int accumulate, gjp_path path, void *stream)
{
    NvtxRange nvtx_range("gjp_adjoint");
    if (!d_volume || !g || !d_proj) return GJP_ERR_INVALID_ARG;
    if (path != GJP_PATH_AUTO && path != GJP_PATH_GATHER && path != GJP_PATH_SLAB && path != GJP_PATH_COMBINE)
        return GJP_ERR_INVALID_ARG;
    int64_t n[3];
    double h[3], o[3];
    gjp_status st = check_grid(nx, ny, nz, voxel_size, volume_origin, n, h, o);
    if (st != GJP_OK) return st;
    if ((st = check_sources(g, n, h, o)) != GJP_OK) return st;
    if (g->n_views > 65535) return GJP_ERR_UNSUPPORTED;
    gjp_cache_entry *entry = nullptr;
    if ((st = get_table(g, n, h, o, &entry)) != GJP_OK) return st;
    const ViewParams *table = entry->d_table;
    cudaStream_t s = (cudaStream_t)stream;
    if (!accumulate) {
        if (cudaMemsetAsync(d_volume, 0, sizeof(float) * (size_t)(n[0] * n[1] * n[2]), s) != cudaSuccess)
            return GJP_ERR_CUDA;
    }
    const bool spl = g->weight == GJP_WEIGHT_SPL;
    if (path == GJP_PATH_SLAB && spl) return GJP_ERR_UNSUPPORTED;   // the slab adjoint implements w_lin only
    if (path == GJP_PATH_COMBINE || (path == GJP_PATH_AUTO && GJP_ADJOINT_AUTO == GJP_PATH_COMBINE)) {
        const VolParams V = make_vol(n, h, g->fov);
        const int n_tv = (g->nv + kTileV - 1) / kTileV;
        const int n_tu = (g->nu + g->tile_u - 1) / g->tile_u;
        const dim3 grid((unsigned)(n_tv * n_tu), (unsigned)g->n_views);
        const dim3 block(kTileV, g->tile_u);
        const int nvw = g->n_views, vgp = launch_view_group(*g, n);
        const bool clip = V.fov_r2 > 0.0f;
        const size_t rows = (size_t)g->tile_u * 32 * sizeof(uint2);   // row tables
#define GJP_COMBINE_LAUNCH(I, S, C)                                                                                \
    gjp_adjoint_combine_kernel<I, S, C><<<grid, block, rows, s>>>(d_proj, V, table, g->nu, g->nv, n_tv, nvw, vgp,   \
                                                                  d_volume)
        if (fits_int32(n)) {
            if (spl) { if (clip) GJP_COMBINE_LAUNCH(int, true, true); else GJP_COMBINE_LAUNCH(int, true, false); }
            else { if (clip) GJP_COMBINE_LAUNCH(int, false, true); else GJP_COMBINE_LAUNCH(int, false, false); }
        } else {
            if (spl) {
                if (clip) GJP_COMBINE_LAUNCH(long long, true, true); else GJP_COMBINE_LAUNCH(long long, true, false);
            } else {
                if (clip) GJP_COMBINE_LAUNCH(long long, false, true); else GJP_COMBINE_LAUNCH(long long, false, false);
            }
        }
#undef GJP_COMBINE_LAUNCH
        return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
    }
    if (path != GJP_PATH_GATHER && !spl) {
        cudaError_t e = cudaSuccess;
        if (try_adjoint_slab(d_proj, n, h, o, *g, *entry, d_volume, s, e))
            return e == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
        if (path == GJP_PATH_SLAB) return GJP_ERR_UNSUPPORTED;
    }
    const VolParams V = make_vol(n, h, g->fov);
    const int n_tv = (g->nv + kTileV - 1) / kTileV;
    const int n_tu = (g->nu + g->tile_u - 1) / g->tile_u;
    const dim3 grid((unsigned)(n_tv * n_tu), (unsigned)g->n_views);
    const dim3 block(kTileV, g->tile_u);
    const int nvw = g->n_views, vgp = launch_view_group(*g, n);
    if (fits_int32(n)) {
        if (spl)
            gjp_adjoint_kernel<int, true><<<grid, block, 0, s>>>(d_proj, V, table, g->nu, g->nv, n_tv, nvw, vgp, d_volume);
        else
            gjp_adjoint_kernel<int, false><<<grid, block, 0, s>>>(d_proj, V, table, g->nu, g->nv, n_tv, nvw, vgp, d_volume);
    } else {
        if (spl)
            gjp_adjoint_kernel<long long, true><<<grid, block, 0, s>>>(d_proj, V, table, g->nu, g->nv, n_tv, nvw, vgp,
                                                                       d_volume);
        else
            gjp_adjoint_kernel<long long, false><<<grid, block, 0, s>>>(d_proj, V, table, g->nu, g->nv, n_tv, nvw, vgp,
                                                                        d_volume);
    }
    return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

gjp_status gjp_adjoint(const float *d_proj, const gjp_geometry *g, int64_t nx, int64_t ny, int64_t nz,
                       const double voxel_size[3], const double volume_origin[3], float *d_volume,
                       int accumulate, void *stream)
{
    return gjp_adjoint_ex(d_proj, g, nx, ny, nz, voxel_size, volume_origin, d_volume, accumulate, GJP_PATH_AUTO,
                          stream);
}

gjp_status gjp_footprint(const gjp_geometry *g, int view, int64_t nx, int64_t ny, int64_t nz,
                         const double voxel_size[3], const double volume_origin[3],
                         unsigned char *d_marks, void *stream)
{
    NvtxRange nvtx_range("gjp_footprint");
    if (!g || !d_marks || view < 0 || view >= g->n_views) return GJP_ERR_INVALID_ARG;
    int64_t n[3];
    double h[3], o[3];
    gjp_status st = check_grid(nx, ny, nz, voxel_size, volume_origin, n, h, o);
    if (st != GJP_OK) return st;
    if ((st = check_sources(g, n, h, o)) != GJP_OK) return st;
    gjp_cache_entry *entry = nullptr;
    if ((st = get_table(g, n, h, o, &entry)) != GJP_OK) return st;
    const ViewParams *table = entry->d_table;
    const VolParams V = make_vol(n, h, g->fov);
    const int n_tv = (g->nv + kTileV - 1) / kTileV;
    const int n_tu = (g->nu + g->tile_u - 1) / g->tile_u;
    const dim3 grid((unsigned)(n_tv * n_tu));
    const dim3 block(kTileV, g->tile_u);
    cudaStream_t s = (cudaStream_t)stream;
    if (fits_int32(n)) gjp_footprint_kernel<int><<<grid, block, 0, s>>>(V, table, view, g->nu, g->nv, n_tv, d_marks);
    else gjp_footprint_kernel<long long><<<grid, block, 0, s>>>(V, table, view, g->nu, g->nv, n_tv, d_marks);
    return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

}  // extern "C"
