// gjp_batch.cu -- many independent GJP forward projections in one
// persistent launch, with a launch-shape autotuner.
//
// A batch holds up to kBatchMaxProblems problems that differ in volume
// size, voxel size, storage type, weight function, view count and detector
// shape.  Every problem is cut into work items -- one detector tile of one
// view -- and all items of all problems form one queue.  A persistent grid
// (resident blocks of every SM, nothing more) takes items from the queue
// with one atomic counter and marches each item's rays with the same
// per-ray code as gjp_forward (Algorithm 1), so a batched projection is
// bitwise equal to the projections made one problem at a time.  Problems
// are queued largest rays first (longest items first, the usual way to keep
// the end of a dynamically scheduled queue short), and a launch is one
// counter reset plus one kernel.  A problem large enough to fill the GPU
// many times over gains nothing from the shared queue: it runs as its own
// launch of the gather forward (with a z-paired copy of a 16-bit volume
// that the batch keeps).  All of these are stream operations, so a stream
// that calls gjp_batch_forward can be captured into a CUDA graph.
//
// The tile shape and the view interleaving of each problem are launch
// choices that change speed, never a result; the paper tunes its CUDA block
// size per configuration, and gjp_batch_autotune does the same per problem
// by timing candidate shapes on a subset of the problem's views.
#include "gjp_common.cuh"

#include <numeric>

namespace gjp_detail {
namespace {

constexpr int kBatchWarps = 4;                       // one block: 4 warps, 128 rays
constexpr int kBatchThreads = kBatchWarps * 32;
constexpr size_t kBatchRowBytes = kBatchWarps * 32 * sizeof(uint2);   // dynamic shared: row tables
constexpr int kBatchMaxProblems = 256;
constexpr int kTuneViews = 24;                       // views timed per autotuner candidate
// A problem with at least this many waves of the persistent grid's blocks
// fills the GPU alone: it runs as its own gather launch (the kernels of
// gjp_forward), not through the shared queue.
constexpr int kSoloWaves = 16;

struct __align__(8) BatchProblem {
    const void *vol;
    float *proj;
    const ViewParams *table;
    VolParams V;
    int nu, nv, n_views;
    int kind;          // dtype (GJP_F32, GJP_BF16, GJP_F16) | 32-bit offsets << 2 | w_spl << 3
    int tile_u;        // detector columns per tile: 1, 2 or 4 (a tile is 128 rays)
    int view_group;    // views interleaved tile by tile
    int n_tu, n_tr;    // tiles along u, along v
    long long items;   // n_views * n_tu * n_tr
};

// One work item: tile `tile` of view `view` (item numbering of block_tile_view).
template <typename T, typename Index, bool SPL>
__device__ __forceinline__ void batch_item(const BatchProblem &P, int tile, int view, int warp, int lane)
{
    const int rows_per_tile = kBatchWarps / P.tile_u;          // 32-row groups per tile
    const int tu = tile / P.n_tr, tr = tile % P.n_tr;
    const int iu = tu * P.tile_u + warp % P.tile_u;
    const int iv = (tr * rows_per_tile + warp / P.tile_u) * 32 + lane;
    const bool active = iu < P.nu && iv < P.nv;
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (!active) return;
    const float val = forward_ray<T, Index, SPL>(static_cast<const T *>(P.vol), P.V, P.table + view, P.nu, P.nv,
                                                 iu, iv, act, warp);
    P.proj[((size_t)view * P.nv + iv) * P.nu + iu] = val;
}

// The kernel is instantiated with only the variants its problems need
// (64-bit offsets, w_spl weights), which keeps its code small.
template <typename T, typename Index, bool ANY_SPL>
__device__ __forceinline__ void batch_item_w(const BatchProblem &P, int tile, int view, int warp, int lane)
{
    if (ANY_SPL && (P.kind & 8)) batch_item<T, Index, ANY_SPL>(P, tile, view, warp, lane);
    else batch_item<T, Index, false>(P, tile, view, warp, lane);
}

template <typename T, bool ANY_I64, bool ANY_SPL>
__device__ __forceinline__ void batch_item_i(const BatchProblem &P, int tile, int view, int warp, int lane)
{
    if (!ANY_I64 || (P.kind & 4)) batch_item_w<T, int, ANY_SPL>(P, tile, view, warp, lane);
    else batch_item_w<T, long long, ANY_SPL>(P, tile, view, warp, lane);
}

// begins[p] = first queue index of problem p, begins[n_probs] = total.
// Each block takes one item at a time from the queue.
template <bool ANY_I64, bool ANY_SPL>
__global__ void __launch_bounds__(kBatchThreads, 8) gjp_batch_forward_kernel(
    const BatchProblem *__restrict__ probs, const long long *__restrict__ begins, int n_probs,
    unsigned long long *__restrict__ counter)
{
    // Everything the loop needs across an item lives in shared memory or
    // kernel parameters, so the march keeps the whole register budget (as
    // in the one-problem kernel) and the item's loads stay in flight.
    __shared__ long long s_begin[kBatchMaxProblems + 1];
    __shared__ long long s_it;                         // the block's item
    __shared__ BatchProblem s_prob;                    // the item's problem
    __shared__ int s_lo, s_new;                        // its index; whether the item starts another problem
    for (int k = threadIdx.x; k <= n_probs; k += blockDim.x) s_begin[k] = begins[k];
    if (threadIdx.x == 0) s_lo = -1;
    for (;;) {
        __syncthreads();                               // the last item's rays are done
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(counter, 1ull);
            s_it = it;
            // the item's problem: found only when it differs from the last
            // item's (queue positions ascend, so a block's items mostly
            // stay in one problem)
            int lo = s_lo;
            const bool fresh = it < s_begin[n_probs] && (lo < 0 || it >= s_begin[lo + 1]);
            if (fresh) {
                int a = 0, b = n_probs - 1;            // last problem with begin <= it
                while (a < b) {
                    const int mid = (a + b + 1) >> 1;
                    if (s_begin[mid] <= it) a = mid;
                    else b = mid - 1;
                }
                lo = a;
            }
            s_lo = lo;
            s_new = fresh ? 1 : 0;
        }
        __syncthreads();
        const long long it = s_it;
        if (it >= s_begin[n_probs]) break;             // queue exhausted (block-uniform)
        const int lo = s_lo;
        if (s_new) {                                   // block-uniform: copy the new problem's record
            constexpr int kWords = (int)(sizeof(BatchProblem) / sizeof(long long));
            if (threadIdx.x < kWords)
                reinterpret_cast<long long *>(&s_prob)[threadIdx.x] =
                    reinterpret_cast<const long long *>(probs + lo)[threadIdx.x];
            __syncthreads();
        }
        const BatchProblem &P = s_prob;
        // item -> (tile, view): block_tile_view's numbering for one problem
        const long long local = it - s_begin[lo];
        const long long n_tiles = (long long)P.n_tu * P.n_tr;
        const long long per = n_tiles * P.view_group;
        const int grp = (int)(local / per);
        const int r = (int)(local - (long long)grp * per);
        const int v0 = grp * P.view_group;
        const int gl = min(P.view_group, P.n_views - v0);
        const int view = v0 + r % gl, tile = r / gl;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        switch (P.kind & 3) {
        case GJP_F32: batch_item_i<float, ANY_I64, ANY_SPL>(P, tile, view, warp, lane); break;
        case GJP_BF16: batch_item_i<__nv_bfloat16, ANY_I64, ANY_SPL>(P, tile, view, warp, lane); break;
        default: batch_item_i<__half, ANY_I64, ANY_SPL>(P, tile, view, warp, lane); break;
        }
    }
}

void shape_problem(BatchProblem &P, int tile_u, int view_group, int n_views)
{
    P.tile_u = tile_u;
    P.view_group = view_group;
    P.n_views = n_views;
    P.n_tu = (P.nu + tile_u - 1) / tile_u;
    const int rows = 32 * (kBatchWarps / tile_u);
    P.n_tr = (P.nv + rows - 1) / rows;
    P.items = (long long)n_views * P.n_tu * P.n_tr;
}

using BatchKernel = void (*)(const BatchProblem *, const long long *, int, unsigned long long *);

BatchKernel batch_kernel(bool any_i64, bool any_spl)
{
    if (any_i64) return any_spl ? gjp_batch_forward_kernel<true, true> : gjp_batch_forward_kernel<true, false>;
    return any_spl ? gjp_batch_forward_kernel<false, true> : gjp_batch_forward_kernel<false, false>;
}

}  // namespace
unsigned batch_tap_faults() { return take_tap_faults(); }

}  // namespace gjp_detail

using namespace gjp_detail;

struct gjp_batch {
    int device = -1;
    int grid = 0;
    BatchKernel kernel = nullptr;
    std::vector<BatchProblem> probs;     // queue order
    std::vector<int> order;              // queue position -> caller's problem index
    std::vector<int> full_views;         // views of each problem (queue order)
    BatchProblem *d_probs = nullptr;
    long long *d_begins = nullptr;
    unsigned long long *d_counter = nullptr;
    BatchProblem *d_tune = nullptr;      // one-problem queue for the autotuner
    long long *d_tune_begins = nullptr;
    std::vector<char> solo;              // per problem (queue order): its own launch
    std::vector<void *> solo_pairs;      // per problem: the z-paired copy of a solo 16-bit problem, or null
    int n_queue = 0;                     // problems in the persistent queue
};

namespace {

gjp_status upload(const BatchProblem *probs, int n, BatchProblem *d_probs, long long *d_begins)
{
    std::vector<long long> begins(n + 1, 0);
    for (int p = 0; p < n; ++p) begins[p + 1] = begins[p] + probs[p].items;
    if (cudaMemcpy(d_probs, probs, sizeof(BatchProblem) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_begins, begins.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess)
        return GJP_ERR_CUDA;
    return GJP_OK;
}

// Uploads the problems that share the persistent queue (the others run alone).
gjp_status upload_queue(gjp_batch *b)
{
    std::vector<BatchProblem> q;
    try {
        for (size_t p = 0; p < b->probs.size(); ++p)
            if (!b->solo[p]) q.push_back(b->probs[p]);
    } catch (const std::bad_alloc &) {
        return GJP_ERR_OOM;
    }
    b->n_queue = (int)q.size();
    return q.empty() ? GJP_OK : upload(q.data(), (int)q.size(), b->d_probs, b->d_begins);
}

gjp_status launch(const gjp_batch *b, const BatchProblem *d_probs, const long long *d_begins, int n,
                  cudaStream_t s)
{
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s) != cudaSuccess) return GJP_ERR_CUDA;
    b->kernel<<<b->grid, kBatchThreads, kBatchRowBytes, s>>>(d_probs, d_begins, n, b->d_counter);
    return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

// One forward of the whole batch: each solo problem as its own gather
// launch (after writing its z-paired copy, if it has one), then one
// persistent launch over the queue.
gjp_status run_batch(const gjp_batch *b, cudaStream_t s)
{
    for (size_t q = 0; q < b->probs.size(); ++q) {
        if (!b->solo[q]) continue;
        const BatchProblem &P = b->probs[q];
        const gjp_dtype dt = (gjp_dtype)(P.kind & 3);
        void *pairs = b->solo_pairs[q];
        if (pairs) {
            const int64_t n[3] = {P.V.n[0], P.V.n[1], P.V.n[2]};
            if (write_zpairs16(P.vol, dt, n, pairs, s) != cudaSuccess) return GJP_ERR_CUDA;
        }
        const GatherShape sh{P.nu, P.nv, P.n_views, P.tile_u, P.view_group, (P.kind & 8) != 0};
        if (forward_gather_shaped(P.vol, dt, P.V, P.table, sh, (P.kind & 4) != 0, P.proj, pairs, s) != cudaSuccess)
            return GJP_ERR_CUDA;
    }
    return b->n_queue > 0 ? launch(b, b->d_probs, b->d_begins, b->n_queue, s) : GJP_OK;
}

void free_batch(gjp_batch *b)
{
    if (!b) return;
    if (b->device >= 0) {
        int cur = -1;
        const bool have = cudaGetDevice(&cur) == cudaSuccess;
        cudaSetDevice(b->device);
        cudaFree(b->d_probs);
        cudaFree(b->d_begins);
        cudaFree(b->d_counter);
        cudaFree(b->d_tune);
        cudaFree(b->d_tune_begins);
        for (void *q : b->solo_pairs) cudaFree(q);
        if (have) cudaSetDevice(cur);
    }
    delete b;
}

bool valid_tile(int t) { return t == 1 || t == 2 || t == 4; }

}  // namespace

extern "C" {

gjp_status gjp_batch_create(const gjp_problem *problems, int count, gjp_batch **out)
{
    NvtxRange nvtx_range("gjp_batch_create");
    if (!out) return GJP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!problems || count < 1 || count > kBatchMaxProblems) return GJP_ERR_INVALID_ARG;
    gjp_batch *b = new (std::nothrow) gjp_batch;
    if (!b) return GJP_ERR_OOM;
    std::vector<BatchProblem> host;
    std::vector<int> planes;
    try {
        host.resize(count);
        planes.resize(count);
    } catch (const std::bad_alloc &) {
        delete b;
        return GJP_ERR_OOM;
    }
    for (int p = 0; p < count; ++p) {
        const gjp_problem &q = problems[p];
        if (!q.d_volume || !q.geometry || !q.d_proj) {
            delete b;
            return GJP_ERR_INVALID_ARG;
        }
        if (q.dtype != GJP_F32 && q.dtype != GJP_BF16 && q.dtype != GJP_F16) {
            delete b;
            return GJP_ERR_INVALID_ARG;
        }
        int64_t n[3];
        double h[3], o[3];
        gjp_status st = check_grid(q.nx, q.ny, q.nz, q.voxel_size, q.has_origin ? q.volume_origin : nullptr, n, h, o);
        if (st == GJP_OK) st = check_sources(q.geometry, n, h, o);
        gjp_cache_entry *entry = nullptr;
        if (st == GJP_OK) st = get_table(q.geometry, n, h, o, &entry);
        if (st != GJP_OK) {
            delete b;
            return st;
        }
        if (b->device < 0 && cudaGetDevice(&b->device) != cudaSuccess) {
            delete b;
            return GJP_ERR_CUDA;
        }
        BatchProblem &P = host[p];
        P.vol = q.d_volume;
        P.proj = q.d_proj;
        P.table = entry->d_table;
        P.V = make_vol(n, h, q.geometry->fov);
        P.nu = q.geometry->nu;
        P.nv = q.geometry->nv;
        P.kind = (int)q.dtype | (fits_int32(n) ? 4 : 0) | (q.geometry->weight == GJP_WEIGHT_SPL ? 8 : 0);
        const int tu = valid_tile(q.geometry->tile_u) ? q.geometry->tile_u : 4;
        shape_problem(P, tu, launch_view_group(*q.geometry, n), q.geometry->n_views);
        planes[p] = (int)std::max(n[0], std::max(n[1], n[2]));
    }
    // queue order: problems with the longest rays (most planes per item) first
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return planes[a] > planes[c]; });
    b->order = order;
    for (int p : order) {
        b->probs.push_back(host[p]);
        b->full_views.push_back(host[p].n_views);
    }
    const size_t pb = sizeof(BatchProblem) * count, bb = sizeof(long long) * (count + 1);
    if (!alloc_gate() || cudaMalloc(&b->d_probs, pb) != cudaSuccess || cudaMalloc(&b->d_begins, bb) != cudaSuccess ||
        cudaMalloc(&b->d_counter, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&b->d_tune, sizeof(BatchProblem)) != cudaSuccess ||
        cudaMalloc(&b->d_tune_begins, 2 * sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return GJP_ERR_OOM;
    }
    bool any_i64 = false, any_spl = false;
    for (const BatchProblem &P : b->probs) {
        any_i64 = any_i64 || !(P.kind & 4);
        any_spl = any_spl || (P.kind & 8);
    }
    b->kernel = batch_kernel(any_i64, any_spl);
    fit_carveout((const void *)b->kernel, kBatchThreads, kBatchRowBytes);
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->kernel, kBatchThreads, kBatchRowBytes) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess || per_sm < 1) {
        free_batch(b);
        return GJP_ERR_CUDA;
    }
    b->grid = per_sm * sms;
    // problems that fill the GPU alone run as their own launch; a 16-bit
    // one reads a z-paired copy kept with the batch where gjp_forward's AUTO
    // would (pairs_pay), unless it cannot be allocated
    try {
        b->solo.assign(count, 0);
        b->solo_pairs.assign(count, nullptr);
    } catch (const std::bad_alloc &) {
        free_batch(b);
        return GJP_ERR_OOM;
    }
    for (int q = 0; q < count; ++q) {
        const BatchProblem &P = b->probs[q];
        if (P.items < (long long)kSoloWaves * b->grid) continue;
        b->solo[q] = 1;
        const int64_t dims[3] = {P.V.n[0], P.V.n[1], P.V.n[2]};
        if ((P.kind & 3) == GJP_F32 || !(P.kind & 4) || !pairs_pay(P.n_views, dims)) continue;
        const size_t bytes = (size_t)P.V.n[0] * P.V.n[1] * P.V.n[2] * sizeof(unsigned);
        if (!alloc_gate() || cudaMalloc(&b->solo_pairs[q], bytes) != cudaSuccess) {
            cudaGetLastError();
            b->solo_pairs[q] = nullptr;
        }
    }
    const gjp_status st = upload_queue(b);
    if (st != GJP_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return GJP_OK;
}

void gjp_batch_destroy(gjp_batch *b) { free_batch(b); }

gjp_status gjp_batch_forward(const gjp_batch *b, void *stream)
{
    NvtxRange nvtx_range("gjp_batch_forward");
    if (!b) return GJP_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GJP_ERR_CUDA;
    if (dev != b->device) return GJP_ERR_INVALID_ARG;
    return run_batch(b, (cudaStream_t)stream);
}

gjp_status gjp_batch_launch_count(const gjp_batch *b, int *launches)
{
    if (!b || !launches) return GJP_ERR_INVALID_ARG;
    int n = b->n_queue > 0 ? 1 : 0;
    for (size_t q = 0; q < b->probs.size(); ++q)
        if (b->solo[q]) n += b->solo_pairs[q] ? 2 : 1;
    *launches = n;
    return GJP_OK;
}

gjp_status gjp_batch_get_tuning(const gjp_batch *b, int problem, int *tile_u, int *view_group)
{
    if (!b || problem < 0 || problem >= (int)b->order.size()) return GJP_ERR_INVALID_ARG;
    for (size_t q = 0; q < b->order.size(); ++q)
        if (b->order[q] == problem) {
            if (tile_u) *tile_u = b->probs[q].tile_u;
            if (view_group) *view_group = b->probs[q].view_group;
            return GJP_OK;
        }
    return GJP_ERR_INTERNAL;
}

gjp_status gjp_batch_set_tuning(gjp_batch *b, int problem, int tile_u, int view_group)
{
    if (!b || problem < 0 || problem >= (int)b->order.size() || !valid_tile(tile_u) || view_group < 1 ||
        view_group > 64)
        return GJP_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GJP_ERR_CUDA;
    if (dev != b->device) return GJP_ERR_INVALID_ARG;
    for (size_t q = 0; q < b->order.size(); ++q)
        if (b->order[q] == problem) shape_problem(b->probs[q], tile_u, view_group, b->full_views[q]);
    return upload_queue(b);
}

gjp_status gjp_batch_autotune(gjp_batch *b, void *stream, int reps)
{
    NvtxRange nvtx_range("gjp_batch_autotune");
    if (!b || reps < 1) return GJP_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GJP_ERR_CUDA;
    if (dev != b->device) return GJP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GJP_ERR_CUDA;
    }
    static const int tiles[] = {1, 2, 4};
    static const int groups[] = {1, 4, 8, 16};
    gjp_status st = GJP_OK;
    // the whole batch, timed as it is now: per-problem shapes that are
    // fastest alone need not be fastest in the shared queue, so the tuned
    // shapes are kept only if the whole batch gets faster
    auto batch_ms = [&](float &out) {
        float ms_min = 3.0e38f;
        for (int r = 0; r <= reps && st == GJP_OK; ++r) {           // r = 0 warms up
            if (cudaEventRecord(e0, s) != cudaSuccess) st = GJP_ERR_CUDA;
            if (st == GJP_OK) st = run_batch(b, s);
            if (st == GJP_OK && cudaEventRecord(e1, s) != cudaSuccess) st = GJP_ERR_CUDA;
            float ms = 0.0f;
            if (st == GJP_OK &&
                (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                st = GJP_ERR_CUDA;
            if (r > 0) ms_min = std::min(ms_min, ms);
        }
        out = ms_min;
    };
    const std::vector<BatchProblem> before = b->probs;
    float ms_before = 0.0f;
    batch_ms(ms_before);
    for (size_t q = 0; q < b->probs.size() && st == GJP_OK; ++q) {
        float best = 3.0e38f;
        int best_t = b->probs[q].tile_u, best_g = b->probs[q].view_group;
        const int nv_t = std::min(b->full_views[q], kTuneViews);
        for (int t : tiles)
            for (int g : groups) {
                BatchProblem P = b->probs[q];
                shape_problem(P, t, g, nv_t);
                if ((st = upload(&P, 1, b->d_tune, b->d_tune_begins)) != GJP_OK) break;
                float ms_min = 3.0e38f;
                for (int r = 0; r <= reps && st == GJP_OK; ++r) {   // r = 0 warms up
                    if (cudaEventRecord(e0, s) != cudaSuccess) st = GJP_ERR_CUDA;
                    if (st == GJP_OK) st = launch(b, b->d_tune, b->d_tune_begins, 1, s);
                    if (st == GJP_OK && cudaEventRecord(e1, s) != cudaSuccess) st = GJP_ERR_CUDA;
                    float ms = 0.0f;
                    if (st == GJP_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                        st = GJP_ERR_CUDA;
                    if (r > 0) ms_min = std::min(ms_min, ms);
                }
                if (st != GJP_OK) break;
                if (ms_min < best) {
                    best = ms_min;
                    best_t = t;
                    best_g = g;
                }
            }
        shape_problem(b->probs[q], best_t, best_g, b->full_views[q]);
    }
    if (st == GJP_OK) st = upload_queue(b);
    float ms_after = 0.0f;
    if (st == GJP_OK) batch_ms(ms_after);
    if (st == GJP_OK && ms_after > ms_before) {                 // keep the shapes it had
        b->probs = before;
        st = upload_queue(b);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // extern "C"
