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

namespace rtsdf {
namespace {

constexpr int SMALL_MAX = 64;   // voxels in a triangle's box handled by one thread

__device__ __forceinline__ long long floor256(long long a) { return a >> 8; }
__device__ __forceinline__ long long ceil256(long long a) { return -((-a) >> 8); }

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

struct TriAxes {
    int lo[3], hi[3];          // clamped voxel range (box-normal axes)
    long long nrm[3];          // triangle normal
    long long nlo, nhi;        // allowed interval of nrm . i
    int ea[9][2];              // the two non-zero components of each edge axis
    int elo[9], ehi[9];        // allowed interval of a . i
};

__device__ __forceinline__ void setup(const int32_t* __restrict__ q, const int32_t* __restrict__ tris,
                                      int64_t t, int n, TriAxes& s) {
    long long v[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int64_t vi = tris[3 * t + k];
#pragma unroll
        for (int a = 0; a < 3; a++) v[k][a] = q[3 * vi + a];
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long mn = min(v[0][a], min(v[1][a], v[2][a]));
        long long mx = max(v[0][a], max(v[1][a], v[2][a]));
        long long l = ceil256(mn - QSUB), h = floor256(mx);
        s.lo[a] = (int)max(l, 0LL);
        s.hi[a] = (int)min(h, (long long)(n - 1));
    }
    long long e[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        e[0][a] = v[1][a] - v[0][a];
        e[1][a] = v[2][a] - v[1][a];
        e[2][a] = v[0][a] - v[2][a];
    }
    s.nrm[0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
    s.nrm[1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
    s.nrm[2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
    {
        long long p = s.nrm[0] * v[0][0] + s.nrm[1] * v[0][1] + s.nrm[2] * v[0][2];
        long long r = (QSUB / 2) * (llabs(s.nrm[0]) + llabs(s.nrm[1]) + llabs(s.nrm[2]));
        long long c = (QSUB / 2) * (s.nrm[0] + s.nrm[1] + s.nrm[2]);
        s.nlo = ceil256(p - r - c);
        s.nhi = floor256(p + r - c);
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            // axis = e_i x unit_j; store the two non-zero components in the
            // order of the voxel coordinates they multiply
            long long ax[3];
            if (j == 0) { ax[0] = 0; ax[1] = e[i][2]; ax[2] = -e[i][1]; }
            else if (j == 1) { ax[0] = -e[i][2]; ax[1] = 0; ax[2] = e[i][0]; }
            else { ax[0] = e[i][1]; ax[1] = -e[i][0]; ax[2] = 0; }
            long long p0 = ax[0] * v[0][0] + ax[1] * v[0][1] + ax[2] * v[0][2];
            long long p1 = ax[0] * v[1][0] + ax[1] * v[1][1] + ax[2] * v[1][2];
            long long p2 = ax[0] * v[2][0] + ax[1] * v[2][1] + ax[2] * v[2][2];
            long long mn = min(p0, min(p1, p2)), mx = max(p0, max(p1, p2));
            long long r = (QSUB / 2) * (llabs(ax[0]) + llabs(ax[1]) + llabs(ax[2]));
            long long c = (QSUB / 2) * (ax[0] + ax[1] + ax[2]);
            const int m = 3 * i + j;
            if (j == 0) { s.ea[m][0] = (int)ax[1]; s.ea[m][1] = (int)ax[2]; }
            else if (j == 1) { s.ea[m][0] = (int)ax[0]; s.ea[m][1] = (int)ax[2]; }
            else { s.ea[m][0] = (int)ax[0]; s.ea[m][1] = (int)ax[1]; }
            s.elo[m] = (int)ceil256(mn - r - c);
            s.ehi[m] = (int)floor256(mx + r - c);
        }
    }
}

__device__ __forceinline__ bool overlaps(const TriAxes& s, int x, int y, int z) {
    long long pn = s.nrm[0] * x + s.nrm[1] * y + s.nrm[2] * z;
    bool ok = (pn >= s.nlo) & (pn <= s.nhi);
#pragma unroll
    for (int m = 0; m < 9; m++) {
        const int j = m % 3;
        // j = 0: (y, z); j = 1: (x, z); j = 2: (x, y)
        int u = j == 0 ? y : x;
        int w = j == 2 ? y : z;
        int p = s.ea[m][0] * u + s.ea[m][1] * w;
        ok &= (p >= s.elo[m]) & (p <= s.ehi[m]);
    }
    return ok;
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
