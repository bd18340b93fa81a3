// gjp_texture.cu -- forward projection through the texture unit.
//
// Two families, both for float32 and float16 volumes (the texture unit has
// no bfloat16 format):
//
//  * GJP_PATH_TEXTURE (exact).  The volume is copied into two layered 2-D
//    texture arrays, one whose layers are the planes x = i (rows y, columns
//    z) and one whose layers are the planes y = i (rows x, columns z).  For
//    a ray driven by x or y, the four taps of Eq. 12 in plane i are one
//    2 x 2 texel footprint of one layer, and one tld4 (texture gather)
//    returns all four; the interpolation weights stay the exact float32
//    values of the gather family (Eq. 10, 13/14), so the results agree with
//    it to float32 rounding.  Border addressing returns zero outside the
//    grid -- the zero-border reading of "p is in volume" -- so every support
//    plane takes the same unchecked path.  Rays driven by z use the global
//    memory march.
//
//  * GJP_PATH_HWLIN (GJP_hwlin of the paper's speed section).  The volume is
//    copied into one 3-D texture with hardware linear filtering, sampled at
//    the plane's integer coordinate plus one half on the driving axis, which
//    makes the filter's weight along m exactly zero, so one filtered fetch is
//    the bilinear interpolation of Eq. 12 in that plane.  The hardware
//    quantises the two fractional weights to 1/256, so this family does not
//    meet the float32 parity tolerance; its measured error is documented and
//    it is never chosen by GJP_PATH_AUTO.
//
// The arrays are cached with the geometry's per-grid device table and
// refilled from the caller's volume on every call (stream ordered), so the
// volume may change between calls; calls of a texture family with the same
// geometry and grid must not overlap on the GPU.
#include "gjp_common.cuh"

namespace gjp_detail {

struct TexCache {
    gjp_dtype dtype = GJP_F32;
    cudaArray_t layered_x = nullptr, layered_y = nullptr, vol3d = nullptr;
    cudaTextureObject_t tex_x = 0, tex_y = 0, tex_3d = 0;
    cudaSurfaceObject_t surf_y = 0;
};

void free_texture_cache(gjp_cache_entry &e)
{
    TexCache *c = static_cast<TexCache *>(e.tex);
    if (!c) return;
    if (c->tex_x) cudaDestroyTextureObject(c->tex_x);
    if (c->tex_y) cudaDestroyTextureObject(c->tex_y);
    if (c->tex_3d) cudaDestroyTextureObject(c->tex_3d);
    if (c->surf_y) cudaDestroySurfaceObject(c->surf_y);
    if (c->layered_x) cudaFreeArray(c->layered_x);
    if (c->layered_y) cudaFreeArray(c->layered_y);
    if (c->vol3d) cudaFreeArray(c->vol3d);
    delete c;
    e.tex = nullptr;
}

namespace {

cudaChannelFormatDesc channel(gjp_dtype t)
{
    return t == GJP_F32 ? cudaCreateChannelDesc<float>() : cudaCreateChannelDescHalf();
}

cudaTextureObject_t make_texture(cudaArray_t a, bool linear)
{
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = a;
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof td);
    td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeBorder;   // zero outside
    td.filterMode = linear ? cudaFilterModeLinear : cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    cudaTextureObject_t t = 0;
    if (cudaCreateTextureObject(&t, &rd, &td, nullptr) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return t;
}

// Copies the C-contiguous [nx][ny][nz] volume into a (layered) array whose
// element (x = k, y = j, layer/depth = i) is vol[i][j][k].
cudaError_t copy_direct(const void *vol, size_t es, const int64_t n[3], cudaArray_t a, cudaStream_t s)
{
    cudaMemcpy3DParms p;
    std::memset(&p, 0, sizeof p);
    p.srcPtr = make_cudaPitchedPtr(const_cast<void *>(vol), (size_t)n[2] * es, (size_t)n[2], (size_t)n[1]);
    p.dstArray = a;
    p.extent = make_cudaExtent((size_t)n[2], (size_t)n[1], (size_t)n[0]);
    p.kind = cudaMemcpyDeviceToDevice;
    return cudaMemcpy3DAsync(&p, s);
}

__device__ __forceinline__ float texel_bits(float v) { return v; }
__device__ __forceinline__ unsigned short texel_bits(__half v) { return __half_as_ushort(v); }

// Layers y = j of the volume: texel (column k, row i, layer j) = vol[i][j][k].
template <typename T>
__global__ void fill_layers_y(const T *__restrict__ vol, int nx, int ny, int nz, cudaSurfaceObject_t surf)
{
    const long long total = (long long)nx * ny * nz;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % nz);
        const long long r = e / nz;
        const int j = (int)(r % ny), i = (int)(r / ny);
        surf2DLayeredwrite(texel_bits(vol[e]), surf, k * (int)sizeof(T), i, j);
    }
}

gjp_status ensure_arrays(gjp_cache_entry &e, gjp_dtype dt, const int64_t n[3], bool hw)
{
    TexCache *c = static_cast<TexCache *>(e.tex);
    if (c && c->dtype != dt) {
        free_texture_cache(e);
        c = nullptr;
    }
    if (!c) {
        c = new (std::nothrow) TexCache;
        if (!c) return GJP_ERR_OOM;
        c->dtype = dt;
        e.tex = c;
    }
    const cudaChannelFormatDesc ch = channel(dt);
    if (hw && !c->vol3d) {
        if (!alloc_gate() ||
            cudaMalloc3DArray(&c->vol3d, &ch, make_cudaExtent((size_t)n[2], (size_t)n[1], (size_t)n[0]), 0) !=
                cudaSuccess) {
            cudaGetLastError();
            c->vol3d = nullptr;
            return GJP_ERR_OOM;
        }
        if (!(c->tex_3d = make_texture(c->vol3d, true))) return GJP_ERR_CUDA;
    }
    if (!hw && !c->layered_x) {
        // planes x = i: (columns z, rows y, layers x); planes y = j: (columns z, rows x, layers y)
        if (!alloc_gate() ||
            cudaMalloc3DArray(&c->layered_x, &ch, make_cudaExtent((size_t)n[2], (size_t)n[1], (size_t)n[0]),
                              cudaArrayLayered) != cudaSuccess ||
            cudaMalloc3DArray(&c->layered_y, &ch, make_cudaExtent((size_t)n[2], (size_t)n[0], (size_t)n[1]),
                              cudaArrayLayered | cudaArraySurfaceLoadStore) != cudaSuccess) {
            cudaGetLastError();
            if (c->layered_x) cudaFreeArray(c->layered_x);
            c->layered_x = c->layered_y = nullptr;
            return GJP_ERR_OOM;
        }
        cudaResourceDesc rd;
        std::memset(&rd, 0, sizeof rd);
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = c->layered_y;
        if (cudaCreateSurfaceObject(&c->surf_y, &rd) != cudaSuccess) {
            cudaGetLastError();
            return GJP_ERR_CUDA;
        }
        if (!(c->tex_x = make_texture(c->layered_x, false)) || !(c->tex_y = make_texture(c->layered_y, false)))
            return GJP_ERR_CUDA;
    }
    return GJP_OK;
}

// Texture x coordinate of a fixed-point position's lower grid point k plus
// one (k >= -1): tld4 at k + 1 fetches texels k and k + 1 (the footprint of
// an unnormalised coordinate c is floor(c - 1/2) and the texel after it).
__device__ __forceinline__ float gather_coord(int k) { return __int_as_float(0x4B000000 | (k + 1)) - 8388608.0f; }

__device__ __forceinline__ float4 tld4_layer(cudaTextureObject_t t, int layer, float x, float y)
{
    float4 r;
    asm("tld4.r.a2d.v4.f32.f32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %8}];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"((unsigned long long)t), "r"(layer), "f"(x), "f"(y), "f"(0.0f));
    return r;
}

// Exact texture-gather forward.  Support planes s_lo .. s_hi of one ray
// driven by x or y; rev marches them downwards (lanes start together).
template <bool SPL>
__device__ __forceinline__ float march_tld4(cudaTextureObject_t t, const Ray &R, bool rev)
{
    const int i0 = rev ? R.s_hi : R.s_lo;
    const int step = rev ? -1 : 1;
    int count = R.s_hi - R.s_lo + 1;
    unsigned long long pa = (unsigned long long)pos_at(R.Pa, R.Ga, i0, R.ic);
    unsigned long long pb = (unsigned long long)pos_at(R.Pb, R.Gb, i0, R.ic);
    const unsigned long long ga = rev ? 0ull - (unsigned long long)R.Ga : (unsigned long long)R.Ga;
    const unsigned long long gb = rev ? 0ull - (unsigned long long)R.Gb : (unsigned long long)R.Gb;
    int layer = i0;
    float acc = 0.0f, part = 0.0f;
    int nb = 0;
    for (; count >= kBatch; count -= kBatch) {
        float4 q[kBatch];
        float da[kBatch], db[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            da[u] = upper_weight<SPL>(frac_of(pa));
            db[u] = upper_weight<SPL>(frac_of(pb));
            q[u] = tld4_layer(t, layer, gather_coord(floor_of(pb)), gather_coord(floor_of(pa)));
            pa += ga;
            pb += gb;
            layer += step;
        }
        float bsum = 0.0f;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            // gather order: (b, a+1), (b+1, a+1), (b+1, a), (b, a) -> v10, v11, v01, v00
            const float e0 = __fmaf_rn(db[u], q[u].z - q[u].w, q[u].w);
            const float e1 = __fmaf_rn(db[u], q[u].y - q[u].x, q[u].x);
            bsum += __fmaf_rn(da[u], e1 - e0, e0);
        }
        part += bsum;
        if ((++nb & 3) == 0) {
            acc += part;
            part = 0.0f;
        }
    }
    acc += part;
    for (; count > 0; --count) {
        const float da = upper_weight<SPL>(frac_of(pa)), db = upper_weight<SPL>(frac_of(pb));
        const float4 q = tld4_layer(t, layer, gather_coord(floor_of(pb)), gather_coord(floor_of(pa)));
        const float e0 = __fmaf_rn(db, q.z - q.w, q.w);
        const float e1 = __fmaf_rn(db, q.y - q.x, q.x);
        acc += __fmaf_rn(da, e1 - e0, e0);
        pa += ga;
        pb += gb;
        layer += step;
    }
    return acc;
}

template <typename T, typename Index, bool SPL>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocksMax) gjp_forward_tld4_kernel(
    cudaTextureObject_t tex_x, cudaTextureObject_t tex_y, const T *__restrict__ vol, VolParams V,
    const ViewParams *__restrict__ views, int nu, int nv, int n_tv, int n_views, int view_group,
    float *__restrict__ proj)
{
    int tile, view;
    block_tile_view(n_views, view_group, tile, view);
    const int iv = (tile % n_tv) * kTileV + threadIdx.x;
    const int iu = (tile / n_tv) * (int)blockDim.y + threadIdx.y;
    const unsigned act = __ballot_sync(0xffffffffu, iv < nv && iu < nu);
    if (iv >= nv || iu >= nu) return;
    ViewParams vp;
    load_view(views, view, vp);
    Ray R;
    setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);
    const unsigned tex_lanes = __ballot_sync(act, R.m != 2);
    float acc;
    if (R.m != 2) {
        // lanes start on a common plane at the end where their supports agree
        const int lo_spread = __reduce_max_sync(tex_lanes, R.s_lo) - __reduce_min_sync(tex_lanes, R.s_lo);
        const int hi_spread = __reduce_max_sync(tex_lanes, R.s_hi) - __reduce_min_sync(tex_lanes, R.s_hi);
        acc = march_tld4<SPL>(R.m == 0 ? tex_x : tex_y, R, hi_spread < lo_spread) * R.step;
    } else {
        const float bsum = march_boundary<T, Index, SPL>(vol, R);
        acc = (march_interior<T, Index, false, SPL>(vol, R) + bsum) * R.step;
    }
    proj[((size_t)view * nv + iv) * nu + iu] = acc;
}

// Hardware-filtered forward (GJP_hwlin).  Texel centres sit at integer +
// 1/2, so sample p (index units) is fetched at p + 1/2 on every axis; the
// driving axis is then an exact integer + 1/2 and its filter weight is 0.
// Positions are affine in the plane index and are formed in float32 per
// sample (their float error, ~1e-4 voxel, is far below the filter's 1/256
// weight steps).
__global__ void __launch_bounds__(kMaxThreads, kMinBlocksMax) gjp_forward_hwlin_kernel(
    cudaTextureObject_t tex, VolParams V, const ViewParams *__restrict__ views, int nu, int nv, int n_tv,
    int n_views, int view_group, float *__restrict__ proj)
{
    int tile, view;
    block_tile_view(n_views, view_group, tile, view);
    const int iv = (tile % n_tv) * kTileV + threadIdx.x;
    const int iu = (tile / n_tv) * (int)blockDim.y + threadIdx.y;
    const unsigned act = __ballot_sync(0xffffffffu, iv < nv && iu < nu);
    if (iv >= nv || iu >= nu) return;
    ViewParams vp;
    load_view(views, view, vp);
    Ray R;
    setup_ray(vp, V, (float)iu - 0.5f * (float)(nu - 1), (float)iv - 0.5f * (float)(nv - 1), R);
    const float inv = 2.3283064365386963e-10f;   // 2^-32
    // c_k(i) = base_k + i * slope_k in texel units (+1/2), for k = x, y, z
    const int a = (R.m == 0) ? 1 : 0;   // the other transverse axis b takes what is left
    const float base_a = __ll2float_rn(R.Pa - (long long)R.ic * R.Ga) * inv + 0.5f;
    const float slope_a = __ll2float_rn(R.Ga) * inv;
    const float base_b = __ll2float_rn(R.Pb - (long long)R.ic * R.Gb) * inv + 0.5f;
    const float slope_b = __ll2float_rn(R.Gb) * inv;
    float base[3], slope[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        base[k] = k == R.m ? 0.5f : (k == a ? base_a : base_b);
        slope[k] = k == R.m ? 1.0f : (k == a ? slope_a : slope_b);
    }
    const int lo_spread = __reduce_max_sync(act, R.s_lo) - __reduce_min_sync(act, R.s_lo);
    const int hi_spread = __reduce_max_sync(act, R.s_hi) - __reduce_min_sync(act, R.s_hi);
    const bool rev = hi_spread < lo_spread;
    float fi = (float)(rev ? R.s_hi : R.s_lo);
    const float fstep = rev ? -1.0f : 1.0f;
    float acc = 0.0f, part = 0.0f;
    int nb = 0;
    int count = R.s_hi - R.s_lo + 1;
    for (; count >= kBatch; count -= kBatch) {
        float v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            // texture x is the volume's z (fastest), y is y, z is x
            v[u] = tex3D<float>(tex, __fmaf_rn(fi, slope[2], base[2]), __fmaf_rn(fi, slope[1], base[1]),
                                __fmaf_rn(fi, slope[0], base[0]));
            fi += fstep;
        }
        part += (v[0] + v[1]) + (v[2] + v[3]);
        if ((++nb & 3) == 0) {
            acc += part;
            part = 0.0f;
        }
    }
    acc += part;
    for (; count > 0; --count) {
        acc += tex3D<float>(tex, __fmaf_rn(fi, slope[2], base[2]), __fmaf_rn(fi, slope[1], base[1]),
                            __fmaf_rn(fi, slope[0], base[0]));
        fi += fstep;
    }
    proj[((size_t)view * nv + iv) * nu + iu] = acc * R.step;
}

}  // namespace

gjp_status forward_texture(const void *d_volume, gjp_dtype dt, const int64_t n[3], const VolParams &V,
                           const gjp_geometry &g, gjp_cache_entry &entry, float *proj, int path, cudaStream_t s)
{
    static_assert(kBatch == 4, "the hwlin batch sum is written for 4 planes");
    if (dt == GJP_BF16) return GJP_ERR_UNSUPPORTED;            // no bfloat16 texture format
    const bool hw = path == GJP_PATH_HWLIN;
    if (hw && g.weight != GJP_WEIGHT_LIN) return GJP_ERR_UNSUPPORTED;   // the filter is w_lin
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GJP_ERR_CUDA;
    int lim[3] = {0, 0, 0};
    const cudaDeviceAttr attrs[2][3] = {
        {cudaDevAttrMaxTexture2DLayeredWidth, cudaDevAttrMaxTexture2DLayeredHeight, cudaDevAttrMaxTexture2DLayeredLayers},
        {cudaDevAttrMaxTexture3DWidth, cudaDevAttrMaxTexture3DHeight, cudaDevAttrMaxTexture3DDepth}};
    for (int k = 0; k < 3; ++k)
        if (cudaDeviceGetAttribute(&lim[k], attrs[hw ? 1 : 0][k], dev) != cudaSuccess) return GJP_ERR_CUDA;
    // hw: (width z, height y, depth x); layered: width z, rows and layers x or y
    if (hw ? (n[2] > lim[0] || n[1] > lim[1] || n[0] > lim[2])
           : (n[2] > lim[0] || std::max(n[0], n[1]) > lim[1] || std::max(n[0], n[1]) > lim[2]))
        return GJP_ERR_UNSUPPORTED;
    const size_t es = dt == GJP_F32 ? 4 : 2;
    gjp_status st;
    {
        std::lock_guard<std::mutex> lock(const_cast<gjp_geometry &>(g).mu);
        st = ensure_arrays(entry, dt, n, hw);
    }
    if (st != GJP_OK) return st;
    TexCache *c = static_cast<TexCache *>(entry.tex);
    const int n_tv = (g.nv + kTileV - 1) / kTileV;
    const int n_tu = (g.nu + g.tile_u - 1) / g.tile_u;
    const dim3 grid((unsigned)(n_tv * n_tu), (unsigned)g.n_views);
    const dim3 block(kTileV, g.tile_u);
    const int nvw = g.n_views, vgp = launch_view_group(g, V.n);
    if (hw) {
        if (copy_direct(d_volume, es, n, c->vol3d, s) != cudaSuccess) return GJP_ERR_CUDA;
        gjp_forward_hwlin_kernel<<<grid, block, 0, s>>>(c->tex_3d, V, entry.d_table, g.nu, g.nv, n_tv, nvw,
                                                               vgp, proj);
        return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
    }
    if (copy_direct(d_volume, es, n, c->layered_x, s) != cudaSuccess) return GJP_ERR_CUDA;
    const long long total = n[0] * n[1] * n[2];
    const int fill_blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    if (dt == GJP_F32)
        fill_layers_y<float><<<fill_blocks, 256, 0, s>>>(static_cast<const float *>(d_volume), (int)n[0],
                                                                 (int)n[1], (int)n[2], c->surf_y);
    else
        fill_layers_y<__half><<<fill_blocks, 256, 0, s>>>(static_cast<const __half *>(d_volume),
                                                                          (int)n[0], (int)n[1], (int)n[2], c->surf_y);
    if (cudaGetLastError() != cudaSuccess) return GJP_ERR_CUDA;
    const bool i32 = fits_int32(n), spl = g.weight == GJP_WEIGHT_SPL;
#define GJP_TLD4_LAUNCH(T, I, S)                                                                                   \
    gjp_forward_tld4_kernel<T, I, S><<<grid, block, 0, s>>>(c->tex_x, c->tex_y, static_cast<const T *>(d_volume), \
                                                            V, entry.d_table, g.nu, g.nv, n_tv, nvw, vgp, proj)
    if (dt == GJP_F32) {
        if (i32) { if (spl) GJP_TLD4_LAUNCH(float, int, true); else GJP_TLD4_LAUNCH(float, int, false); }
        else { if (spl) GJP_TLD4_LAUNCH(float, long long, true); else GJP_TLD4_LAUNCH(float, long long, false); }
    } else {
        if (i32) { if (spl) GJP_TLD4_LAUNCH(__half, int, true); else GJP_TLD4_LAUNCH(__half, int, false); }
        else { if (spl) GJP_TLD4_LAUNCH(__half, long long, true); else GJP_TLD4_LAUNCH(__half, long long, false); }
    }
#undef GJP_TLD4_LAUNCH
    return cudaGetLastError() == cudaSuccess ? GJP_OK : GJP_ERR_CUDA;
}

unsigned texture_tap_faults() { return take_tap_faults(); }

}  // namespace gjp_detail
