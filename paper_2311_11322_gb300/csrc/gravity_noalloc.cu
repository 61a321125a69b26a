// gravity_noalloc.cu -- softened direct-sum gravity of one set of spheres
// that allocates no memory at all.
//
// Who needs it: code that may not call cudaMalloc or any allocator -- for
// example a caller running inside someone else's memory pool or arena with a
// fixed budget, a real-time or safety-certified host loop where allocation
// after start-up is forbidden, or a plugin whose host application owns every
// device allocation.  Such a caller cannot create a dem_world (a world
// obtains its buffers at add time), but it can hand this entry point device
// buffers it already owns for the inputs and the output.
//
// The formula is the world's gravity formula (FP32 pair terms, FP64 sums;
// results agree with the world's within the mixed-precision tolerance, not
// bitwise, since the world sums symmetric tile pairs), with the j range
// split into kNAChunks parts: each part writes an FP64 partial sum per sphere,
// and a second kernel adds the parts in a fixed order.  Those partial sums are
// the only scratch memory, and here they live in the file-scope array
// g_na_scratch below (16 MiB), which the CUDA runtime places in device memory
// when the library is loaded; every GPU that loads the library keeps it until
// the process exits.  Host code cannot use g_na_scratch's name as a device
// address: the host-side symbol is only a stand-in, and a kernel handed it
// would fault or, where the GPU can reach host memory, silently use the wrong
// memory.  The device address is therefore looked up with
// cudaGetSymbolAddress, once per device, with that device current, on the
// first call made on it.
#include <cstdio>
#include <mutex>

#include "dem_internal.h"

namespace {

constexpr int kNAChunks = 4;                 // j-range parts
constexpr int kNAMaxSpheres = 131072;        // largest n accepted
constexpr int kNABlock = 128;
constexpr int kNAFlush = 1024;
constexpr int kNAMaxDevices = 64;

// 4 parts x 131,072 spheres x 32 B = 16 MiB of partial sums.
static __device__ __align__(256) dem::dbl4 g_na_scratch[kNAChunks * kNAMaxSpheres];

std::mutex g_na_mutex;
dem::dbl4 *g_na_addr[kNAMaxDevices] = {nullptr};

__global__ void __launch_bounds__(kNABlock)
k_na_partial(const float4 *__restrict__ pm, const int32_t *__restrict__ agg, int n, int jc,
             float eps2, dem::dbl4 *scratch)
{
    __shared__ float4 sp[kNABlock];
    __shared__ int sa[kNABlock];
    const int i = blockIdx.x * kNABlock + threadIdx.x;
    const int c = blockIdx.y;
    const int j0 = c * jc;
    const int j1 = min(n, j0 + jc);
    const float4 xi = i < n ? pm[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int ai = i < n ? agg[i] : -2;
    float ax = 0.f, ay = 0.f, az = 0.f;
    double dx = 0.0, dy = 0.0, dz = 0.0;
    int since = 0;
    for (int jt = j0; jt < j1; jt += kNABlock) {
        __syncthreads();
        const int j = jt + threadIdx.x;
        if (j < j1) {
            sp[threadIdx.x] = pm[j];
            sa[threadIdx.x] = agg[j];
        } else {
            sp[threadIdx.x] = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f);
            sa[threadIdx.x] = -1;
        }
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < kNABlock; ++jj) {
            const float4 pj = sp[jj];
            const float ddx = pj.x - xi.x, ddy = pj.y - xi.y, ddz = pj.z - xi.z;
            const float r2 = fmaf(ddz, ddz, fmaf(ddy, ddy, fmaf(ddx, ddx, eps2)));
            const float inv = rsqrtf(r2);
            float s = (pj.w * inv) * (inv * inv);
            // same aggregate (and i itself): skipped; with eps = 0 two coincident
            // spheres of different aggregates exert no force on each other
            s = (sa[jj] == ai || !(r2 > 0.f)) ? 0.f : s;
            ax = fmaf(ddx, s, ax);
            ay = fmaf(ddy, s, ay);
            az = fmaf(ddz, s, az);
        }
        since += kNABlock;
        if (since >= kNAFlush) {
            since = 0;
            dx += ax; dy += ay; dz += az;
            ax = ay = az = 0.f;
        }
    }
    // every (part, sphere) slot read by k_na_combine is written here in the
    // same call, so nothing left over from an earlier call is ever read
    if (i < n) scratch[(size_t)c * kNAMaxSpheres + i] = dem::make_dbl4(dx + ax, dy + ay, dz + az, 0.0);
}

__global__ void k_na_combine(const double *__restrict__ mass, int n, double G,
                             const dem::dbl4 *__restrict__ scratch, dem::dbl4 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int c = 0; c < kNAChunks; ++c) {
        const dem::dbl4 v = scratch[(size_t)c * kNAMaxSpheres + i];
        sx += v.x; sy += v.y; sz += v.z;
    }
    const double gm = G * mass[i];
    out[i] = dem::make_dbl4(gm * sx, gm * sy, gm * sz, 0.0);
}

void set_msg(char *msg, size_t len, const char *text)
{
    if (msg && len) snprintf(msg, len, "%s", text);
}

}  // namespace

extern "C" dem_status dem_gravity_noalloc(const void *pos_mass, const double *mass,
                                          const int32_t *agg_id, int32_t n, double G,
                                          double eps_soft, double *force_out, void *cuda_stream,
                                          char *msg, size_t msg_len)
{
    set_msg(msg, msg_len, "");
    if (!pos_mass || !mass || !agg_id || !force_out) {
        set_msg(msg, msg_len, "dem_gravity_noalloc: NULL pointer argument");
        return DEM_ERR_ARG;
    }
    if (n < 1 || n > kNAMaxSpheres) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "dem_gravity_noalloc: n = %d outside 1..%d (the fixed scratch holds %d spheres)",
                 n, kNAMaxSpheres, kNAMaxSpheres);
        set_msg(msg, msg_len, buf);
        return DEM_ERR_ARG;
    }
    if (!(G >= 0.0) || !(eps_soft >= 0.0) || !(G < 1e300) || !(eps_soft < 1e300)) {
        set_msg(msg, msg_len, "dem_gravity_noalloc: G and eps_soft must be finite and >= 0");
        return DEM_ERR_ARG;
    }
    if ((((uintptr_t)pos_mass) & 15) || (((uintptr_t)force_out) & 31) || (((uintptr_t)mass) & 7) ||
        (((uintptr_t)agg_id) & 3)) {
        set_msg(msg, msg_len, "dem_gravity_noalloc: pos_mass must be 16-byte, force_out 32-byte, "
                              "mass 8-byte and agg_id 4-byte aligned");
        return DEM_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNAMaxDevices) {
        set_msg(msg, msg_len, "dem_gravity_noalloc: no usable current CUDA device");
        return DEM_ERR_CUDA;
    }
    dem::dbl4 *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess || !p) {
                char buf[200];
                snprintf(buf, sizeof buf, "dem_gravity_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                set_msg(msg, msg_len, buf);
                return DEM_ERR_CUDA;
            }
            g_na_addr[dev] = (dem::dbl4 *)p;
        }
        scratch = g_na_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int jc = (n + kNAChunks - 1) / kNAChunks;
    dim3 grid((n + kNABlock - 1) / kNABlock, kNAChunks);
    k_na_partial<<<grid, kNABlock, 0, st>>>((const float4 *)pos_mass, agg_id, n, jc,
                                            (float)(eps_soft * eps_soft), scratch);
    k_na_combine<<<(n + 255) / 256, 256, 0, st>>>(mass, n, G, scratch, (dem::dbl4 *)force_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[200];
        snprintf(buf, sizeof buf, "dem_gravity_noalloc: launch failed: %s", cudaGetErrorString(e));
        set_msg(msg, msg_len, buf);
        return DEM_ERR_CUDA;
    }
    return DEM_OK;
}
