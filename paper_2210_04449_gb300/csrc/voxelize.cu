// Sec. 2.1 -- conservative voxelization of the scene into the coarse grid.
//
// The paper rasterizes the scene three times (orthographic views along +x,
// +y, +z, depth writes off).  Rasterization samples fragment centres and can
// miss thin or sliver triangles, so this kernel instead marks every voxel
// whose closed cube meets a closed triangle.  Vertices are quantised to
// 1/256 voxel (fp32 subtract and multiply, round half to even) and the
// overlap is decided by the separating-axis theorem (box normals, the
// triangle normal, the nine edge x box-axis directions) in exact integer
// arithmetic, so the result does not depend on evaluation order.
//
// Per triangle, every axis a is reduced to an integer interval of a . i
// (i = voxel index) outside which the voxel is separated:
//   a . centre(i) = 256 (a . i) + 128 (a_x + a_y + a_z)
//   separated  <=>  a . centre < min_k a . q_k - r_a  or  > max_k a . q_k + r_a,
//   r_a = 128 (|a_x| + |a_y| + |a_z|),
// so the inner voxel loop only evaluates a . i and two compares per axis.
#include "internal.cuh"
#include "vox_dev.cuh"

namespace rtsdf {
namespace {

using namespace dev;

__global__ void k_quantise(const float* __restrict__ verts, int64_t nv, float bx, float by, float bz,
                           float scale, int n, int32_t* __restrict__ q, uint32_t* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv * 3) return;
    const int a = (int)(i % 3);
    const float b = a == 0 ? bx : (a == 1 ? by : bz);
    const float lo = -(float)(QSUB / 2) * (float)n;
    const float hi = (float)(3 * QSUB / 2) * (float)n;
    float v = __fmul_rn(__fsub_rn(verts[i], b), scale);
    if (!(v >= lo && v <= hi)) {
        atomicOr(err, ERR_MESH);
        v = (v >= lo) ? hi : lo;   // NaN and -inf go to lo
        if (!(v == v)) v = lo;
    }
    q[i] = __float2int_rn(v);
}

__global__ void k_validate_tris(int32_t* __restrict__ tris, int64_t nt, int64_t nv, uint32_t* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt * 3) return;
    int32_t t = tris[i];
    if (t < 0 || t >= nv) {
        atomicOr(err, ERR_MESH);
        tris[i] = 0;
    }
}

__global__ void __launch_bounds__(128) k_voxelize_small(const int32_t* __restrict__ q,
                                                       const int32_t* __restrict__ tris, int64_t nt,
                                                       int n, uint32_t* __restrict__ seeds,
                                                       int32_t* __restrict__ big_list,
                                                       uint32_t* __restrict__ big_count) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    TriAxes s;
    setup(q, tris, t, n, s);
    int cx = s.hi[0] - s.lo[0] + 1, cy = s.hi[1] - s.lo[1] + 1, cz = s.hi[2] - s.lo[2] + 1;
    if (cx <= 0 || cy <= 0 || cz <= 0) return;
    if ((long long)cx * cy * cz > SMALL_MAX) {
        uint32_t slot = atomicAdd(big_count, 1u);
        big_list[slot] = (int32_t)t;
        return;
    }
    for (int z = s.lo[2]; z <= s.hi[2]; z++)
        for (int y = s.lo[1]; y <= s.hi[1]; y++)
            for (int x = s.lo[0]; x <= s.hi[0]; x++)
                if (overlaps(s, x, y, z))
                    seeds[x + (size_t)n * (y + (size_t)n * z)] = pack_seed(x, y, z);
}

// One block per large triangle (grid-stride over the list); the threads of a
// block split the triangle's voxel box.
__global__ void __launch_bounds__(256) k_voxelize_big(const int32_t* __restrict__ q,
                                                     const int32_t* __restrict__ tris,
                                                     const int32_t* __restrict__ big_list,
                                                     const uint32_t* __restrict__ big_count, int n,
                                                     uint32_t* __restrict__ seeds) {
    const uint32_t nb = *big_count;
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        TriAxes s;
        setup(q, tris, big_list[b], n, s);
        const int cx = s.hi[0] - s.lo[0] + 1, cy = s.hi[1] - s.lo[1] + 1, cz = s.hi[2] - s.lo[2] + 1;
        const long long total = (long long)cx * cy * cz;
        for (long long i = threadIdx.x; i < total; i += blockDim.x) {
            int x = s.lo[0] + (int)(i % cx);
            int y = s.lo[1] + (int)((i / cx) % cy);
            int z = s.lo[2] + (int)(i / ((long long)cx * cy));
            if (overlaps(s, x, y, z)) seeds[x + (size_t)n * (y + (size_t)n * z)] = pack_seed(x, y, z);
        }
    }
}

}  // namespace

cudaError_t launch_quantise(rtsdf_ctx* c) {
    if (c->nv == 0) return cudaSuccess;
    const float scale = (float)(c->nc * QSUB) / c->cfg.extent;
    int64_t m = c->nv * 3;
    RTSDF_LAUNCH(c, k_quantise, (unsigned)((m + 255) / 256), 256, 0, c->verts, c->nv, c->cfg.bmin[0],
                 c->cfg.bmin[1], c->cfg.bmin[2], scale, c->nc, c->qverts, c->d_err);
    return cudaGetLastError();
}

cudaError_t launch_validate_tris(rtsdf_ctx* c) {
    if (c->nt == 0) return cudaSuccess;
    int64_t m = c->nt * 3;
    RTSDF_LAUNCH(c, k_validate_tris, (unsigned)((m + 255) / 256), 256, 0, c->tris, c->nt, c->nv, c->d_err);
    return cudaGetLastError();
}

cudaError_t launch_voxelize(rtsdf_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->seeds[0], 0xFF, c->nc3 * sizeof(uint32_t), c->stream);
    if (e != cudaSuccess) return e;
    c->cur = 0;
    if (c->nt == 0) return cudaSuccess;
    e = cudaMemsetAsync(c->d_big_count, 0, sizeof(uint32_t), c->stream);
    if (e != cudaSuccess) return e;
    RTSDF_LAUNCH(c, k_voxelize_small, (unsigned)((c->nt + 127) / 128), 128, 0, c->qverts, c->tris, c->nt,
                 c->nc, c->seeds[0], c->big_list, c->d_big_count);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    RTSDF_LAUNCH(c, k_voxelize_big, (unsigned)(sms > 0 ? sms * 4 : 512), 256, 0, c->qverts, c->tris,
                 c->big_list, c->d_big_count, c->nc, c->seeds[0]);
    return cudaGetLastError();
}

}  // namespace rtsdf
