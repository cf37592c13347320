// Device helpers of the conservative voxelization (Sec. 2.1), shared by the
// per-scene kernels (voxelize.cu) and the batched persistent kernel.
#pragma once

#include "internal.cuh"

namespace rtsdf {
namespace dev {

constexpr int SMALL_MAX = 64;   // voxels in a triangle's box handled by one thread

__device__ __forceinline__ long long floor256(long long a) { return a >> 8; }
__device__ __forceinline__ long long ceil256(long long a) { return -((-a) >> 8); }

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

}  // namespace dev
}  // namespace rtsdf
