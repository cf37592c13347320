/*
 * RTSDF CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, slow restatement of the method of "RTSDF: Generating Signed
 * Distance Fields in Real Time for Soft Shadow Rendering" (Tan, Chua, Koh,
 * Bhojan; Pacific Graphics 2020 work-in-progress paper):
 *
 *   Sec. 2.1  scene voxelization and 3D jump flooding -> coarse SDF,
 *   Sec. 2.2  near-surface random-direction ray tracing, Eq. 1 accumulation
 *             and the front/back hit vote for the sign,
 *   Sec. 2.3  sphere-traced soft-shadow visibility from the fine SDF,
 *
 * plus the reverse-mode derivative of the Sec. 2.3 march.  Only the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header, table or constant
 * generator with the CUDA implementation.
 *
 * Precision: fp64, except where a floating-point result decides an integer
 * result -- the voxel quantisation (Sec. 2.1), the ray direction, the
 * ray/triangle hit decision, the closest-hit argmin and the front/back vote
 * (Sec. 2.2) -- which are taken in fp32 with the operation order written out
 * below (explicit fmaf, no contraction: compile with -ffp-contract=off).
 *
 * Grids are stored x-fastest: linear index = x + n*(y + n*z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

/* ======================================================================
 * Sec. 2.1 -- voxelization.
 * The paper rasterizes three orthographic views with depth writes off.
 * Here a voxel is occupied iff the closed triangle meets the closed voxel
 * cube (a conservative voxelization).  Vertices are first quantised to
 * 1/256 of a coarse voxel (fp32 subtract, fp32 multiply, round half to
 * even); the overlap test is then the separating-axis test of
 * Akenine-Moller (2001) -- box face normals, triangle normal, and the nine
 * edge x box-axis directions -- evaluated exactly in int64.
 * ====================================================================== */

#define ORC_SUB 256   /* quantisation steps per coarse voxel */

static int64_t floordiv64(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

static int64_t iabs64(int64_t a) { return a < 0 ? -a : a; }

/* r: triangle vertices relative to the box centre; hh: box half size. */
static int tri_box_overlap_i64(const int64_t r[3][3], int64_t hh)
{
    for (int a = 0; a < 3; a++) {
        int64_t mn = r[0][a], mx = r[0][a];
        for (int k = 1; k < 3; k++) {
            if (r[k][a] < mn) mn = r[k][a];
            if (r[k][a] > mx) mx = r[k][a];
        }
        if (mn > hh || mx < -hh) return 0;
    }
    int64_t e[3][3];
    for (int a = 0; a < 3; a++) {
        e[0][a] = r[1][a] - r[0][a];
        e[1][a] = r[2][a] - r[1][a];
        e[2][a] = r[0][a] - r[2][a];
    }
    /* triangle plane */
    int64_t nrm[3] = {
        e[0][1] * e[1][2] - e[0][2] * e[1][1],
        e[0][2] * e[1][0] - e[0][0] * e[1][2],
        e[0][0] * e[1][1] - e[0][1] * e[1][0],
    };
    int64_t dpl = nrm[0] * r[0][0] + nrm[1] * r[0][1] + nrm[2] * r[0][2];
    int64_t rad = hh * (iabs64(nrm[0]) + iabs64(nrm[1]) + iabs64(nrm[2]));
    if (dpl > rad || dpl < -rad) return 0;
    /* edge x unit-axis directions */
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) {
            int64_t ax[3];
            if (j == 0) { ax[0] = 0; ax[1] = e[i][2]; ax[2] = -e[i][1]; }
            else if (j == 1) { ax[0] = -e[i][2]; ax[1] = 0; ax[2] = e[i][0]; }
            else { ax[0] = e[i][1]; ax[1] = -e[i][0]; ax[2] = 0; }
            int64_t p0 = ax[0] * r[0][0] + ax[1] * r[0][1] + ax[2] * r[0][2];
            int64_t p1 = ax[0] * r[1][0] + ax[1] * r[1][1] + ax[2] * r[1][2];
            int64_t p2 = ax[0] * r[2][0] + ax[1] * r[2][1] + ax[2] * r[2][2];
            int64_t mn = p0 < p1 ? p0 : p1; if (p2 < mn) mn = p2;
            int64_t mx = p0 > p1 ? p0 : p1; if (p2 > mx) mx = p2;
            int64_t ra = hh * (iabs64(ax[0]) + iabs64(ax[1]) + iabs64(ax[2]));
            if (mn > ra || mx < -ra) return 0;
        }
    }
    return 1;
}

/* Quantise one coordinate; returns 0 when it lies outside the accepted
 * range [bmin - extent/2, bmin + 3*extent/2] (in grid units: [-n/2, 3n/2]
 * voxels) or is not finite. */
static int quantise(float p, float b, float scale, int n, int64_t* q)
{
    float v = (p - b) * scale;
    float lo = -(float)(ORC_SUB / 2) * (float)n, hi = (float)(3 * ORC_SUB / 2) * (float)n;
    if (!(v >= lo && v <= hi)) return 0;
    *q = (int64_t)rintf(v);
    return 1;
}

/* Scale from world units to quantisation steps: (n*256)/extent in fp32. */
EXPORT float orc_quant_scale(int n, float extent) { return (float)(n * ORC_SUB) / extent; }

/* Quantise all vertices (fp32 decision, see header).  q: int64 [nv*3].
 * Returns 0, or -1 on a non-finite / out-of-range vertex. */
EXPORT int orc_quantise_vertices(const float* verts, int64_t nv, const float* bmin,
                                 float extent, int n, int64_t* q)
{
    float scale = orc_quant_scale(n, extent);
    for (int64_t i = 0; i < nv; i++)
        for (int a = 0; a < 3; a++)
            if (!quantise(verts[3 * i + a], bmin[a], scale, n, &q[3 * i + a])) return -1;
    return 0;
}

/* occ: int32 [n^3]; occ[v] = v where some triangle touches voxel v, else -1.
 * Returns 0; -1 on a bad vertex; -2 on a triangle index out of range. */
EXPORT int orc_voxelize(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                        const float* bmin, float extent, int n, int32_t* occ)
{
    int64_t n3 = (int64_t)n * n * n;
    for (int64_t v = 0; v < n3; v++) occ[v] = -1;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(nv > 0 ? nv : 1));
    if (orc_quantise_vertices(verts, nv, bmin, extent, n, q) != 0) { free(q); return -1; }
    for (int64_t t = 0; t < nt; t++)
        for (int k = 0; k < 3; k++)
            if (tris[3 * t + k] < 0 || tris[3 * t + k] >= nv) { free(q); return -2; }
    const int64_t hh = ORC_SUB / 2;
    for (int64_t t = 0; t < nt; t++) {
        int64_t p[3][3];
        for (int k = 0; k < 3; k++)
            for (int a = 0; a < 3; a++) p[k][a] = q[3 * (int64_t)tris[3 * t + k] + a];
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            int64_t mn = p[0][a], mx = p[0][a];
            for (int k = 1; k < 3; k++) {
                if (p[k][a] < mn) mn = p[k][a];
                if (p[k][a] > mx) mx = p[k][a];
            }
            lo[a] = floordiv64(mn, ORC_SUB) - 1;
            hi[a] = floordiv64(mx, ORC_SUB);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > n - 1) hi[a] = n - 1;
        }
        for (int64_t z = lo[2]; z <= hi[2]; z++)
            for (int64_t y = lo[1]; y <= hi[1]; y++)
                for (int64_t x = lo[0]; x <= hi[0]; x++) {
                    int64_t c[3] = {x * ORC_SUB + hh, y * ORC_SUB + hh, z * ORC_SUB + hh};
                    int64_t r[3][3];
                    for (int k = 0; k < 3; k++)
                        for (int a = 0; a < 3; a++) r[k][a] = p[k][a] - c[a];
                    if (tri_box_overlap_i64(r, hh)) {
                        int64_t v = x + (int64_t)n * (y + (int64_t)n * z);
                        occ[v] = (int32_t)v;
                    }
                }
    }
    free(q);
    return 0;
}

/* Exact overlap test of one quantised triangle against one voxel (for
 * tests that probe single pairs). */
EXPORT int orc_tri_voxel_overlap(const int64_t* qtri /* [9] */, int x, int y, int z)
{
    const int64_t hh = ORC_SUB / 2;
    int64_t c[3] = {(int64_t)x * ORC_SUB + hh, (int64_t)y * ORC_SUB + hh, (int64_t)z * ORC_SUB + hh};
    int64_t r[3][3];
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 3; a++) r[k][a] = qtri[3 * k + a] - c[a];
    return tri_box_overlap_i64(r, hh);
}

/* ======================================================================
 * Sec. 2.1 -- jump flooding with the occupied voxels as seeds.
 * Step lengths 2^(ceil(log2 n)-1), ..., 2, 1 (ceil(log2 n) passes).  In each
 * pass every voxel v looks at the 27 voxels v + {-k,0,k}^3 that lie inside
 * the grid, reads their current nearest-seed entry from the previous pass
 * (Jacobi: a pass reads only the previous pass's grid), and keeps the seed
 * with the smallest squared distance to v, ties going to the smaller
 * linear seed index.  Seeds are linear voxel indices, -1 = none.
 * ====================================================================== */

static int ceil_log2(int n)
{
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}

EXPORT int orc_jfa_passes(int n) { return ceil_log2(n); }

EXPORT int orc_jfa(const int32_t* init, int n, int32_t* out)
{
    int64_t n3 = (int64_t)n * n * n;
    int32_t* a = (int32_t*)malloc(sizeof(int32_t) * (size_t)n3);
    int32_t* b = (int32_t*)malloc(sizeof(int32_t) * (size_t)n3);
    memcpy(a, init, sizeof(int32_t) * (size_t)n3);
    int L = ceil_log2(n), passes = 0;
    for (int k = L > 0 ? (1 << (L - 1)) : 0; k >= 1; k >>= 1) {
        #pragma omp parallel for schedule(static)
        for (int z = 0; z < n; z++)
            for (int y = 0; y < n; y++)
                for (int x = 0; x < n; x++) {
                    int32_t best = -1;
                    int64_t bestd = INT64_MAX;
                    for (int dz = -k; dz <= k; dz += k)
                        for (int dy = -k; dy <= k; dy += k)
                            for (int dx = -k; dx <= k; dx += k) {
                                int nx = x + dx, ny = y + dy, nz = z + dz;
                                if (nx < 0 || ny < 0 || nz < 0 || nx >= n || ny >= n || nz >= n) continue;
                                int32_t s = a[nx + (int64_t)n * (ny + (int64_t)n * nz)];
                                if (s < 0) continue;
                                int64_t sx = s % n, sy = (s / n) % n, sz = s / ((int64_t)n * n);
                                int64_t d2 = (sx - x) * (sx - x) + (sy - y) * (sy - y) + (sz - z) * (sz - z);
                                if (d2 < bestd || (d2 == bestd && s < best)) { bestd = d2; best = s; }
                            }
                    b[x + (int64_t)n * (y + (int64_t)n * z)] = best;
                }
        int32_t* t = a; a = b; b = t;
        passes++;
    }
    memcpy(out, a, sizeof(int32_t) * (size_t)n3);
    free(a);
    free(b);
    return passes;
}

/* Squared distance from each voxel to its assigned seed (-1 when none). */
EXPORT void orc_seed_d2(const int32_t* seeds, int n, int64_t* d2)
{
    int64_t n3 = (int64_t)n * n * n;
    for (int64_t v = 0; v < n3; v++) {
        int32_t s = seeds[v];
        if (s < 0) { d2[v] = -1; continue; }
        int64_t x = v % n, y = (v / n) % n, z = v / ((int64_t)n * n);
        int64_t sx = s % n, sy = (s / n) % n, sz = s / ((int64_t)n * n);
        d2[v] = (sx - x) * (sx - x) + (sy - y) * (sy - y) + (sz - z) * (sz - z);
    }
}

/* Pin: exact squared distance to the nearest seed over ALL seeds (brute
 * force, O(n^3 * seeds)); -1 when there are no seeds. */
EXPORT void orc_edt_brute(const int32_t* init, int n, int64_t* d2)
{
    int64_t n3 = (int64_t)n * n * n, ns = 0;
    int64_t* sx = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n3 > 0 ? n3 : 1));
    for (int64_t v = 0; v < n3; v++)
        if (init[v] >= 0) {
            sx[3 * ns] = v % n; sx[3 * ns + 1] = (v / n) % n; sx[3 * ns + 2] = v / ((int64_t)n * n);
            ns++;
        }
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t v = 0; v < n3; v++) {
        int64_t x = v % n, y = (v / n) % n, z = v / ((int64_t)n * n), best = -1;
        for (int64_t i = 0; i < ns; i++) {
            int64_t dx = sx[3 * i] - x, dy = sx[3 * i + 1] - y, dz = sx[3 * i + 2] - z;
            int64_t d = dx * dx + dy * dy + dz * dz;
            if (best < 0 || d < best) best = d;
        }
        d2[v] = best;
    }
    free(sx);
}

/* Pin: exact squared Euclidean distance transform by separable lower
 * envelopes of parabolas (Felzenszwalb & Huttenlocher, "Distance Transforms
 * of Sampled Functions", 2012), one 1D transform per axis.  -1 when no seed. */
static void edt_1d(const double* f, int n, double* d, int* v, double* zb)
{
    int k = 0;
    int first = -1;
    for (int q = 0; q < n; q++) if (f[q] < INFINITY) { first = q; break; }
    if (first < 0) { for (int q = 0; q < n; q++) d[q] = INFINITY; return; }
    v[0] = first;
    zb[0] = -INFINITY;
    zb[1] = INFINITY;
    for (int q = first + 1; q < n; q++) {
        if (!(f[q] < INFINITY)) continue;
        double s;
        for (;;) {
            int p = v[k];
            s = ((f[q] + (double)q * q) - (f[p] + (double)p * p)) / (2.0 * (q - p));
            if (s <= zb[k] && k > 0) { k--; continue; }
            break;
        }
        if (s <= zb[k]) { /* k == 0: the new parabola dominates everywhere */
            v[0] = q; zb[0] = -INFINITY; zb[1] = INFINITY; continue;
        }
        k++;
        v[k] = q;
        zb[k] = s;
        zb[k + 1] = INFINITY;
    }
    k = 0;
    for (int q = 0; q < n; q++) {
        while (zb[k + 1] < q) k++;
        double dq = (double)q - v[k];
        d[q] = dq * dq + f[v[k]];
    }
}

EXPORT void orc_edt_separable(const int32_t* init, int n, int64_t* d2)
{
    int64_t n3 = (int64_t)n * n * n;
    double* g = (double*)malloc(sizeof(double) * (size_t)n3);
    for (int64_t i = 0; i < n3; i++) g[i] = init[i] >= 0 ? 0.0 : INFINITY;
    for (int axis = 0; axis < 3; axis++) {
        #pragma omp parallel
        {
            double* f = (double*)malloc(sizeof(double) * n);
            double* d = (double*)malloc(sizeof(double) * n);
            int* v = (int*)malloc(sizeof(int) * n);
            double* zb = (double*)malloc(sizeof(double) * (n + 1));
            #pragma omp for schedule(static)
            for (int64_t line = 0; line < (int64_t)n * n; line++) {
                int64_t a = line % n, b = line / n, base, stride;
                if (axis == 0) { base = (int64_t)n * (a + (int64_t)n * b); stride = 1; }
                else if (axis == 1) { base = a + (int64_t)n * n * b; stride = n; }
                else { base = a + (int64_t)n * b; stride = (int64_t)n * n; }
                for (int q = 0; q < n; q++) f[q] = g[base + q * stride];
                edt_1d(f, n, d, v, zb);
                for (int q = 0; q < n; q++) g[base + q * stride] = d[q];
            }
            free(f); free(d); free(v); free(zb);
        }
    }
    for (int64_t i = 0; i < n3; i++) d2[i] = g[i] < INFINITY ? (int64_t)g[i] : -1;
    free(g);
}

/* ======================================================================
 * Sec. 2.2 -- random ray directions from a counter-based generator.
 * Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * S-box style word permutation, the key bumped by the Weyl constants after
 * each round.  The 4x64 variant uses the same round structure with 64-bit
 * words; it is exported so the structure can be checked against an
 * independent library implementation.
 * ====================================================================== */

#define PHILOX_DEFINE(NAME, T, TT, SHIFT, M0, M1, W0, W1)                       \
    EXPORT void NAME(const T* ctr, const T* key, T* out)                        \
    {                                                                           \
        T c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];                   \
        T k0 = key[0], k1 = key[1];                                             \
        for (int r = 0; r < 10; r++) {                                          \
            TT p0 = (TT)(M0) * (TT)c0;                                          \
            TT p1 = (TT)(M1) * (TT)c2;                                          \
            T hi0 = (T)(p0 >> SHIFT), lo0 = (T)p0;                              \
            T hi1 = (T)(p1 >> SHIFT), lo1 = (T)p1;                              \
            T n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;       \
            c0 = n0; c1 = n1; c2 = n2; c3 = n3;                                 \
            k0 = (T)(k0 + (T)(W0));                                             \
            k1 = (T)(k1 + (T)(W1));                                             \
        }                                                                       \
        out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;                     \
    }

PHILOX_DEFINE(orc_philox4x32_10, uint32_t, uint64_t, 32,
              0xD2511F53u, 0xCD9E8D57u, 0x9E3779B9u, 0xBB67AE85u)
PHILOX_DEFINE(orc_philox4x64_10, uint64_t, unsigned __int128, 64,
              0xD2E7470EE14C6C93ull, 0xCA5A826395121157ull,
              0x9E3779B97F4A7C15ull, 0xBB67AE8584CAA73Bull)

/* A uniform direction on the unit sphere for (texel, frame, ray): Marsaglia
 * (1972).  Counter = (draw, ray, frame, texel), key = (seed lo, seed hi).
 * Each draw yields two candidate pairs; a pair (a, b) uses the top 23 bits
 * of two words as odd integers A, B in (-2^23, 2^23), a = A 2^-23.  It is
 * accepted when A^2 + B^2 < 2^46 (exact integer test, i.e. a^2 + b^2 < 1);
 * then with s = a^2 + b^2 the direction is
 *   (2a sqrt(1-s), 2b sqrt(1-s), 1 - 2s).
 * After 8 draws without acceptance the direction is (0, 0, 1).
 * fp32 (the decision precision, see header): s = (float)(A^2+B^2) * 2^-46. */
EXPORT int orc_sphere_dir(uint64_t seed, uint32_t texel, uint32_t frame, uint32_t ray, float* d)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t draw = 0; draw < 8; draw++) {
        uint32_t ctr[4] = {draw, ray, frame, texel}, w[4];
        orc_philox4x32_10(ctr, key, w);
        for (int p = 0; p < 2; p++) {
            int32_t A = 2 * (int32_t)(w[2 * p] >> 9) + 1 - (1 << 23);
            int32_t B = 2 * (int32_t)(w[2 * p + 1] >> 9) + 1 - (1 << 23);
            int64_t S = (int64_t)A * A + (int64_t)B * B;
            if (S < ((int64_t)1 << 46)) {
                float s = (float)S * 0x1p-46f;
                float root = sqrtf(1.0f - s);
                float a = (float)A * 0x1p-23f, b = (float)B * 0x1p-23f;
                d[0] = (2.0f * a) * root;
                d[1] = (2.0f * b) * root;
                d[2] = 1.0f - 2.0f * s;
                return (int)(2 * draw + p + 1);
            }
        }
    }
    d[0] = 0.0f; d[1] = 0.0f; d[2] = 1.0f;
    return 0;
}

/* ======================================================================
 * Sec. 2.2 -- closest hit of one ray: Moller & Trumbore (1997) ray/triangle
 * test in fp32 (the decision precision), closed triangles, t >= 0.
 *   e1 = v1 - v0, e2 = v2 - v0, P = D x e2, det = e1 . P  (det == 0: miss)
 *   inv = 1/det, T = O - v0, u = (T . P) inv  in [0, 1]
 *   Q = T x e1, v = (D . Q) inv >= 0, u + v <= 1, t = (e2 . Q) inv >= 0
 * dot(a, b)   = fma(a.z, b.z, fma(a.y, b.y, a.x * b.x))
 * cross(a,b).x = fma(a.y, b.z, -(a.z * b.y)) (and cyclically).
 * det > 0  <=>  D . (e1 x e2) < 0: the ray meets the front (outward) face.
 * ====================================================================== */

static inline float dot3f(const float* a, const float* b)
{
    return fmaf(a[2], b[2], fmaf(a[1], b[1], a[0] * b[0]));
}

static inline void cross3f(const float* a, const float* b, float* c)
{
    c[0] = fmaf(a[1], b[2], -(a[2] * b[1]));
    c[1] = fmaf(a[2], b[0], -(a[0] * b[2]));
    c[2] = fmaf(a[0], b[1], -(a[1] * b[0]));
}

static int ray_tri_f32(const float* o, const float* d, const float* v0, const float* e1,
                       const float* e2, float* t, int* front)
{
    float p[3];
    cross3f(d, e2, p);
    float det = dot3f(e1, p);
    if (det == 0.0f) return 0;
    float inv = 1.0f / det;
    float tv[3] = {o[0] - v0[0], o[1] - v0[1], o[2] - v0[2]};
    float u = dot3f(tv, p) * inv;
    if (!(u >= 0.0f && u <= 1.0f)) return 0;
    float q[3];
    cross3f(tv, e1, q);
    float v = dot3f(d, q) * inv;
    if (!(v >= 0.0f && u + v <= 1.0f)) return 0;
    float tt = dot3f(e2, q) * inv;
    if (!(tt >= 0.0f)) return 0;
    *t = tt;
    *front = det > 0.0f;
    return 1;
}

/* One ray against one triangle (pins). Returns hit; t, front out. */
EXPORT int orc_ray_triangle(const float* o, const float* d, const float* v0, const float* v1,
                            const float* v2, float* t, int* front)
{
    float e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
    float e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
    return ray_tri_f32(o, d, v0, e1, e2, t, front);
}

/* Closest hit over ALL triangles (brute force, ascending index so equal t
 * keeps the smaller triangle index).  Returns the triangle index or -1. */
static int64_t closest_hit(const float* o, const float* d, const float* tv0, const float* te1,
                           const float* te2, int64_t nt, float* tbest, int* fbest)
{
    int64_t best = -1;
    float bt = INFINITY;
    int bf = 0;
    for (int64_t i = 0; i < nt; i++) {
        float t;
        int f;
        if (ray_tri_f32(o, d, tv0 + 3 * i, te1 + 3 * i, te2 + 3 * i, &t, &f) && t < bt) {
            bt = t; bf = f; best = i;
        }
    }
    *tbest = bt;
    *fbest = bf;
    return best;
}

static void tri_edges(const float* verts, const int32_t* tris, int64_t nt, float* tv0, float* te1, float* te2)
{
    for (int64_t i = 0; i < nt; i++) {
        const float* a = verts + 3 * (int64_t)tris[3 * i];
        const float* b = verts + 3 * (int64_t)tris[3 * i + 1];
        const float* c = verts + 3 * (int64_t)tris[3 * i + 2];
        for (int k = 0; k < 3; k++) {
            tv0[3 * i + k] = a[k];
            te1[3 * i + k] = b[k] - a[k];
            te2[3 * i + k] = c[k] - a[k];
        }
    }
}

/* Fine texel centre in fp32: bmin + (j + 0.5) * (extent / nf). */
EXPORT void orc_texel_centre(const float* bmin, float extent, int nf, int64_t j, float* o)
{
    float hf = extent / (float)nf;
    int64_t jx = j % nf, jy = (j / nf) % nf, jz = j / ((int64_t)nf * nf);
    o[0] = bmin[0] + ((float)jx + 0.5f) * hf;
    o[1] = bmin[1] + ((float)jy + 0.5f) * hf;
    o[2] = bmin[2] + ((float)jz + 0.5f) * hf;
}

/* One frame of tracing for a list of fine texels: r_t (smallest closest-hit
 * distance over the R rays, +inf when no ray hit) and the numbers of rays
 * whose closest hit was a front / back face.  Also returns per-texel the
 * index of the ray and triangle that gave r_t (-1 when none). */
EXPORT void orc_trace(const float* verts, const int32_t* tris, int64_t nt, const float* bmin,
                      float extent, int nf, uint64_t seed, int frame, int R,
                      const int64_t* texels, int64_t m, float* rmin, int32_t* nfront,
                      int32_t* nback, int64_t* best_tri,
                      int32_t* min_back /* face of the nearest hit (1 = back), ties -> front; may be NULL */)
{
    float* tv0 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te1 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te2 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    tri_edges(verts, tris, nt, tv0, te1, te2);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; i++) {
        float o[3];
        orc_texel_centre(bmin, extent, nf, texels[i], o);
        float r = INFINITY;
        int32_t cf = 0, cb = 0, rb = 0;
        int64_t bt = -1;
        for (int ray = 0; ray < R; ray++) {
            float d[3], t;
            int f;
            orc_sphere_dir(seed, (uint32_t)texels[i], (uint32_t)frame, (uint32_t)ray, d);
            int64_t hit = closest_hit(o, d, tv0, te1, te2, nt, &t, &f);
            if (hit < 0) continue;
            if (f) cf++; else cb++;
            if (t < r) { r = t; bt = hit; rb = !f; }
            else if (t == r && f) rb = 0;   /* equal nearest distance: a front hit wins */
        }
        rmin[i] = r;
        nfront[i] = cf;
        nback[i] = cb;
        if (best_tri) best_tri[i] = bt;
        if (min_back) min_back[i] = rb;
    }
    free(tv0); free(te1); free(te2);
}

/* Closest hit of arbitrary rays (fp32 decision) -- t (+inf on miss), front flag, triangle. */
EXPORT void orc_cast_rays(const float* verts, const int32_t* tris, int64_t nt, const float* orig,
                          const float* dirs, int64_t nr, float* tout, int32_t* front, int64_t* tri)
{
    float* tv0 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te1 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te2 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    tri_edges(verts, tris, nt, tv0, te1, te2);
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nr; i++) {
        float t;
        int f;
        int64_t h = closest_hit(orig + 3 * i, dirs + 3 * i, tv0, te1, te2, nt, &t, &f);
        tout[i] = t;
        front[i] = h >= 0 ? f : 0;
        tri[i] = h;
    }
    free(tv0); free(te1); free(te2);
}

/* ======================================================================
 * Sec. 2.2 -- the same closest hit, found faster (for whole-frame checks).
 * A bounding-volume hierarchy only skips triangles that a ray cannot reach
 * before its best hit; every triangle it does test goes through the same
 * fp32 ray_tri_f32 and the same (t, then smaller index) rule, so the result
 * is the brute-force closest_hit's.  Build: median split (by centroid,
 * fp64, ties by triangle index) along the longest axis of the centroid
 * bounds, leaves of at most ORC_LEAF triangles.  Boxes are fp64 over the
 * fp32 vertices, widened by ORC_PAD on every side, and a box is entered
 * when the ray's fp64 slab interval meets [0, best t + ORC_PAD]; the pad
 * keeps a triangle that fp32 rounding accepts slightly outside its exact
 * extent (a grazing hit) from being skipped.  The tests compare this path
 * with the brute-force one bit for bit.
 * ====================================================================== */

#define ORC_LEAF 4
#define ORC_PAD 1e-4

typedef struct {
    double lo[3], hi[3];
    int64_t left, right;      /* children (internal) or -1 */
    int64_t first, count;     /* leaf: range of the index array */
} obvh_node;

typedef struct {
    obvh_node* nodes;
    int64_t n_nodes;
    int64_t* idx;             /* triangle index per leaf slot */
    double* cen;              /* centroid [nt][3] */
    const float* tv0; const float* te1; const float* te2;
    const float* verts; const int32_t* tris;
} obvh;

static double cen_key(const obvh* b, int64_t i, int ax) { return b->cen[3 * i + ax]; }

/* strict order on (centroid along ax, triangle index) */
static int cen_less(const obvh* b, int64_t i, int64_t j, int ax)
{
    double a = cen_key(b, i, ax), c = cen_key(b, j, ax);
    return a < c || (a == c && i < j);
}

/* quickselect: reorder idx[lo..hi) so that idx[k] is the k-th smallest and
 * every element before it is smaller */
static void select_k(const obvh* b, int64_t* idx, int64_t lo, int64_t hi, int64_t k, int ax)
{
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        /* median of three as the pivot */
        int64_t a = idx[lo], m = idx[mid], z = idx[hi - 1], pv;
        if (cen_less(b, a, m, ax)) pv = cen_less(b, m, z, ax) ? m : (cen_less(b, a, z, ax) ? z : a);
        else pv = cen_less(b, a, z, ax) ? a : (cen_less(b, m, z, ax) ? z : m);
        int64_t i = lo, j = hi - 1;
        while (i <= j) {
            while (cen_less(b, idx[i], pv, ax)) i++;
            while (cen_less(b, pv, idx[j], ax)) j--;
            if (i <= j) { int64_t t = idx[i]; idx[i] = idx[j]; idx[j] = t; i++; j--; }
        }
        if (k <= j) hi = j + 1;
        else if (k >= i) lo = i;
        else return;
    }
}

static void obvh_box(const obvh* b, int64_t first, int64_t count, double* lo, double* hi)
{
    for (int a = 0; a < 3; a++) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    for (int64_t s = first; s < first + count; s++) {
        int64_t t = b->idx[s];
        for (int v = 0; v < 3; v++) {
            const float* p = b->verts + 3 * (int64_t)b->tris[3 * t + v];
            for (int a = 0; a < 3; a++) {
                if ((double)p[a] < lo[a]) lo[a] = p[a];
                if ((double)p[a] > hi[a]) hi[a] = p[a];
            }
        }
    }
    for (int a = 0; a < 3; a++) { lo[a] -= ORC_PAD; hi[a] += ORC_PAD; }
}

static int64_t obvh_build_rec(obvh* b, int64_t first, int64_t count)
{
    int64_t id = b->n_nodes++;
    obvh_node* nd = &b->nodes[id];
    obvh_box(b, first, count, nd->lo, nd->hi);
    nd->first = first;
    nd->count = count;
    nd->left = nd->right = -1;
    if (count <= ORC_LEAF) return id;
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t s = first; s < first + count; s++)
        for (int a = 0; a < 3; a++) {
            double c = cen_key(b, b->idx[s], a);
            if (c < clo[a]) clo[a] = c;
            if (c > chi[a]) chi[a] = c;
        }
    int ax = 0;
    for (int a = 1; a < 3; a++) if (chi[a] - clo[a] > chi[ax] - clo[ax]) ax = a;
    int64_t half = count / 2;
    select_k(b, b->idx, first, first + count, first + half, ax);
    int64_t l = obvh_build_rec(b, first, half);
    int64_t r = obvh_build_rec(b, first + half, count - half);
    b->nodes[id].left = l;   /* nodes[] does not move: sized up front */
    b->nodes[id].right = r;
    return id;
}

static void obvh_build(obvh* b, const float* verts, const int32_t* tris, int64_t nt,
                       const float* tv0, const float* te1, const float* te2)
{
    b->verts = verts; b->tris = tris; b->tv0 = tv0; b->te1 = te1; b->te2 = te2;
    b->nodes = (obvh_node*)malloc(sizeof(obvh_node) * (size_t)(2 * (nt > 0 ? nt : 1)));
    b->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
    b->cen = (double*)malloc(sizeof(double) * 3 * (size_t)(nt > 0 ? nt : 1));
    b->n_nodes = 0;
    for (int64_t i = 0; i < nt; i++) {
        b->idx[i] = i;
        for (int a = 0; a < 3; a++) {
            double s = 0;
            for (int v = 0; v < 3; v++) s += verts[3 * (int64_t)tris[3 * i + v] + a];
            b->cen[3 * i + a] = s / 3.0;
        }
    }
    if (nt > 0) obvh_build_rec(b, 0, nt);
}

static void obvh_free(obvh* b) { free(b->nodes); free(b->idx); free(b->cen); }

/* Entry distance of the ray (fp64, origin o, reciprocal direction inv;
 * inv = +-inf on a zero component) into the box within [0, tmax], or -1
 * when it misses. */
static double obvh_box_entry(const obvh_node* n, const double* o, const double* d, const double* inv, double tmax)
{
    double t0 = 0.0, t1 = tmax;
    for (int a = 0; a < 3; a++) {
        if (d[a] == 0.0) {
            if (o[a] < n->lo[a] || o[a] > n->hi[a]) return -1.0;
            continue;
        }
        double ta = (n->lo[a] - o[a]) * inv[a], tb = (n->hi[a] - o[a]) * inv[a];
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return -1.0;
    }
    return t0;
}

#define OBVH_STACK 128

/* Stack traversal, nearer child first; a popped node is skipped when its
 * entry distance exceeds the best hit found since it was pushed (plus the
 * pad). */
static int64_t obvh_closest_hit(const obvh* b, const float* o, const float* d, float* tbest, int* fbest)
{
    int64_t best = -1;
    float bt = INFINITY;
    int bf = 0;
    if (b->n_nodes == 0) { *tbest = bt; *fbest = bf; return best; }
    double od[3] = {o[0], o[1], o[2]}, dd[3] = {d[0], d[1], d[2]};
    double inv[3];
    for (int a = 0; a < 3; a++) inv[a] = dd[a] != 0.0 ? 1.0 / dd[a] : INFINITY;
    int64_t stack[OBVH_STACK];
    double entry[OBVH_STACK];
    int sp = 0;
    if (obvh_box_entry(&b->nodes[0], od, dd, inv, INFINITY) < 0.0) { *tbest = bt; *fbest = bf; return best; }
    stack[sp] = 0;
    entry[sp++] = 0.0;
    while (sp > 0) {
        sp--;
        const obvh_node* n = &b->nodes[stack[sp]];
        if (entry[sp] > (double)bt + ORC_PAD) continue;
        if (n->left < 0) {
            for (int64_t s = n->first; s < n->first + n->count; s++) {
                int64_t i = b->idx[s];
                float t;
                int f;
                if (ray_tri_f32(o, d, b->tv0 + 3 * i, b->te1 + 3 * i, b->te2 + 3 * i, &t, &f) &&
                    (t < bt || (t == bt && i < best))) {
                    bt = t; bf = f; best = i;
                }
            }
            continue;
        }
        double tmax = (double)bt + ORC_PAD;   /* +inf while nothing was hit */
        double el = obvh_box_entry(&b->nodes[n->left], od, dd, inv, tmax);
        double er = obvh_box_entry(&b->nodes[n->right], od, dd, inv, tmax);
        if (sp + 2 > OBVH_STACK) abort();   /* depth is about log2(nt): never */
        int64_t first = n->left, second = n->right;
        double ef = el, es = er;
        if (er >= 0.0 && (el < 0.0 || er < el)) { first = n->right; second = n->left; ef = er; es = el; }
        if (es >= 0.0) { stack[sp] = second; entry[sp++] = es; }
        if (ef >= 0.0) { stack[sp] = first; entry[sp++] = ef; }
    }
    *tbest = bt;
    *fbest = bf;
    return best;
}

/* orc_trace with the closest hit of every ray found through the hierarchy
 * above (same outputs, same arithmetic). */
EXPORT void orc_trace_bvh(const float* verts, const int32_t* tris, int64_t nt, const float* bmin,
                          float extent, int nf, uint64_t seed, int frame, int R,
                          const int64_t* texels, int64_t m, float* rmin, int32_t* nfront,
                          int32_t* nback, int64_t* best_tri, int32_t* min_back)
{
    float* tv0 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te1 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te2 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    tri_edges(verts, tris, nt, tv0, te1, te2);
    obvh b;
    obvh_build(&b, verts, tris, nt, tv0, te1, te2);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; i++) {
        float o[3];
        orc_texel_centre(bmin, extent, nf, texels[i], o);
        float r = INFINITY;
        int32_t cf = 0, cb = 0, rb = 0;
        int64_t bt = -1;
        for (int ray = 0; ray < R; ray++) {
            float d[3], t;
            int f;
            orc_sphere_dir(seed, (uint32_t)texels[i], (uint32_t)frame, (uint32_t)ray, d);
            int64_t hit = obvh_closest_hit(&b, o, d, &t, &f);
            if (hit < 0) continue;
            if (f) cf++; else cb++;
            if (t < r) { r = t; bt = hit; rb = !f; }
            else if (t == r && f) rb = 0;   /* equal nearest distance: a front hit wins */
        }
        rmin[i] = r;
        nfront[i] = cf;
        nback[i] = cb;
        if (best_tri) best_tri[i] = bt;
        if (min_back) min_back[i] = rb;
    }
    obvh_free(&b);
    free(tv0); free(te1); free(te2);
}

/* orc_cast_rays through the hierarchy. */
EXPORT void orc_cast_rays_bvh(const float* verts, const int32_t* tris, int64_t nt, const float* orig,
                              const float* dirs, int64_t nr, float* tout, int32_t* front, int64_t* tri)
{
    float* tv0 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te1 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te2 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    tri_edges(verts, tris, nt, tv0, te1, te2);
    obvh b;
    obvh_build(&b, verts, tris, nt, tv0, te1, te2);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nr; i++) {
        float t;
        int f;
        int64_t h = obvh_closest_hit(&b, orig + 3 * i, dirs + 3 * i, &t, &f);
        tout[i] = t;
        front[i] = h >= 0 ? f : 0;
        tri[i] = h;
    }
    obvh_free(&b);
    free(tv0); free(te1); free(te2);
}

/* ======================================================================
 * Pin only: exact unsigned distance from points to a triangle mesh, fp64.
 * Closest point on a triangle by Voronoi-region classification (Ericson,
 * Real-Time Collision Detection, Sec. 5.1.5), brute force over triangles.
 * ====================================================================== */

static void closest_pt_tri(const double* p, const double* a, const double* b, const double* c, double* out)
{
    double ab[3], ac[3], ap[3];
    for (int k = 0; k < 3; k++) { ab[k] = b[k] - a[k]; ac[k] = c[k] - a[k]; ap[k] = p[k] - a[k]; }
#define DOT(u, v) ((u)[0] * (v)[0] + (u)[1] * (v)[1] + (u)[2] * (v)[2])
    double d1 = DOT(ab, ap), d2 = DOT(ac, ap);
    if (d1 <= 0 && d2 <= 0) { memcpy(out, a, 3 * sizeof(double)); return; }
    double bp[3];
    for (int k = 0; k < 3; k++) bp[k] = p[k] - b[k];
    double d3 = DOT(ab, bp), d4 = DOT(ac, bp);
    if (d3 >= 0 && d4 <= d3) { memcpy(out, b, 3 * sizeof(double)); return; }
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0 && d1 >= 0 && d3 <= 0) {
        double v = d1 / (d1 - d3);
        for (int k = 0; k < 3; k++) out[k] = a[k] + v * ab[k];
        return;
    }
    double cp[3];
    for (int k = 0; k < 3; k++) cp[k] = p[k] - c[k];
    double d5 = DOT(ab, cp), d6 = DOT(ac, cp);
    if (d6 >= 0 && d5 <= d6) { memcpy(out, c, 3 * sizeof(double)); return; }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0 && d2 >= 0 && d6 <= 0) {
        double w = d2 / (d2 - d6);
        for (int k = 0; k < 3; k++) out[k] = a[k] + w * ac[k];
        return;
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
        double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int k = 0; k < 3; k++) out[k] = b[k] + w * (c[k] - b[k]);
        return;
    }
    double den = 1.0 / (va + vb + vc);
    double v = vb * den, w = vc * den;
    for (int k = 0; k < 3; k++) out[k] = a[k] + ab[k] * v + ac[k] * w;
#undef DOT
}

EXPORT void orc_point_mesh_distance(const float* verts, const int32_t* tris, int64_t nt,
                                    const double* pts, int64_t np, double* dist)
{
    #pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < np; i++) {
        double best = INFINITY;
        for (int64_t t = 0; t < nt; t++) {
            double a[3], b[3], c[3], q[3];
            for (int k = 0; k < 3; k++) {
                a[k] = verts[3 * (int64_t)tris[3 * t] + k];
                b[k] = verts[3 * (int64_t)tris[3 * t + 1] + k];
                c[k] = verts[3 * (int64_t)tris[3 * t + 2] + k];
            }
            closest_pt_tri(pts + 3 * i, a, b, c, q);
            double dx = q[0] - pts[3 * i], dy = q[1] - pts[3 * i + 1], dz = q[2] - pts[3 * i + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (d < best) best = d;
        }
        dist[i] = best;
    }
}

/* ======================================================================
 * Sec. 2.3 -- soft-shadow visibility by sphere tracing the fine SDF, fp64.
 * S(q): trilinear interpolation of the cell-centred grid (centre of texel j
 * at bmin + (j + 0.5) h), coordinates clamped to the first/last centre.
 * Per shading point p with normal nrm and unit light direction L:
 *   o = p + 2 eps nrm, t = 0, res = 1, ph = 1e20
 *   for i < steps:
 *     q = o + t L; stop if q leaves [bmin, bmin + extent]^3
 *     h = S(q); if h < eps: visibility 0 (the march hit a surface)
 *     y = h^2 / (2 ph), dd = sqrt(max(h^2 - y^2, 0))
 *     if t - y > 0 and k dd / (t - y) < res: res = k dd / (t - y)
 *     ph = h; t += min(h, step_max)
 *   visibility = clamp(res, 0, 1)
 * The penumbra estimate k dd / (t - y) combines the current and the
 * previous sample as in Aaltonen (2018), the estimate Sec. 2.3 adopts;
 * step_max is the restricted maximum step of Sec. 2.3.
 * ====================================================================== */

typedef struct {
    int64_t idx[8];
    double w[8];
    double dw[8][3];   /* d w / d q */
} tri_taps;

static double trilinear(const float* f, int n, const double* bmin, double h, const double* q, tri_taps* tp)
{
    int64_t i0[3], i1[3];
    double fr[3], dg[3];
    for (int a = 0; a < 3; a++) {
        double g = (q[a] - bmin[a]) / h - 0.5;
        double gc = g;
        dg[a] = 1.0 / h;
        if (!(gc > 0.0)) { gc = 0.0; dg[a] = 0.0; }
        if (gc >= (double)(n - 1)) { gc = (double)(n - 1); dg[a] = 0.0; }
        int64_t b = (int64_t)floor(gc);
        if (b > n - 2) b = n - 2;
        if (b < 0) b = 0;
        i0[a] = b;
        i1[a] = n > 1 ? b + 1 : 0;
        fr[a] = n > 1 ? gc - (double)b : 0.0;
    }
    double val = 0.0;
    int c = 0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++, c++) {
                int64_t x = dx ? i1[0] : i0[0], y = dy ? i1[1] : i0[1], z = dz ? i1[2] : i0[2];
                double wx = dx ? fr[0] : 1 - fr[0], wy = dy ? fr[1] : 1 - fr[1], wz = dz ? fr[2] : 1 - fr[2];
                int64_t id = x + (int64_t)n * (y + (int64_t)n * z);
                double w = wx * wy * wz;
                val += w * (double)f[id];
                if (tp) {
                    tp->idx[c] = id;
                    tp->w[c] = w;
                    tp->dw[c][0] = (dx ? 1.0 : -1.0) * wy * wz * dg[0];
                    tp->dw[c][1] = wx * (dy ? 1.0 : -1.0) * wz * dg[1];
                    tp->dw[c][2] = wx * wy * (dz ? 1.0 : -1.0) * dg[2];
                }
            }
    return val;
}

EXPORT double orc_sample(const float* f, int n, const double* bmin, double extent, const double* q)
{
    return trilinear(f, n, bmin, extent / n, q, NULL);
}

typedef struct {
    int n;
    double h, extent, eps, k, step_max;
    int steps;
    const double* bmin;
} march_cfg;

static int inside_box(const double* q, const double* bmin, double extent)
{
    for (int a = 0; a < 3; a++)
        if (!(q[a] >= bmin[a] && q[a] <= bmin[a] + extent)) return 0;
    return 1;
}

/* Forward march of one point; records per step (t_i, h_i) when arrays given.
 * Returns visibility; *nstep = samples taken, *argmin = step that set res
 * (-1 if none), *term = 1 if stopped by h < eps. */
/* Relative closeness of two values that a decision compares. */
static double rel_gap(double a, double b, double scale)
{
    return fabs(a - b) / scale;
}

static double march_one(const float* f, const march_cfg* mc, const double* p, const double* nrm,
                        const double* L, double shift, double* ts, double* hs, int* nstep, int* argmin,
                        int* term, double* margin)
{
    /* shift: the origin's jitter toward the light (Sec. 2.3), world units.
     * margin (may be NULL): the smallest relative gap, over the whole march,
     * between the two sides of any discrete decision (inside the volume,
     * h < eps, t - y > 0, a new minimum, h < step_max, the root's argument
     * > 0); a march with a large margin takes the same path under small
     * perturbations of its inputs or rounding. */
    double o[3];
    for (int a = 0; a < 3; a++) o[a] = p[a] + 2.0 * mc->eps * nrm[a] + shift * L[a];
    double t = 0.0, res = 1.0, ph = 1e20;
    double mg = INFINITY;
    int am = -1, i;
    *term = 0;
    for (i = 0; i < mc->steps; i++) {
        double q[3] = {o[0] + t * L[0], o[1] + t * L[1], o[2] + t * L[2]};
        if (margin)
            for (int a = 0; a < 3; a++) {
                double lo = rel_gap(q[a], mc->bmin[a], mc->h), hi = rel_gap(q[a], mc->bmin[a] + mc->extent, mc->h);
                if (lo < mg) mg = lo;
                if (hi < mg) mg = hi;
            }
        if (!inside_box(q, mc->bmin, mc->extent)) break;
        double h = trilinear(f, mc->n, mc->bmin, mc->h, q, NULL);
        if (ts) { ts[i] = t; hs[i] = h; }
        if (margin) {
            double g1 = rel_gap(h, mc->eps, mc->eps);
            if (g1 < mg) mg = g1;
        }
        if (h < mc->eps) { *term = 1; *nstep = i + 1; *argmin = am; if (margin) *margin = mg; return 0.0; }
        double y = h * h / (2.0 * ph);
        double a2 = h * h - y * y;
        double dd = sqrt(a2 > 0.0 ? a2 : 0.0);
        if (margin) {
            /* at t = 0 (the first step) t - y > 0 is false at any precision */
            double g2 = t > 0.0 ? rel_gap(t, y, mc->h) : INFINITY;
            double g3 = rel_gap(a2, 0.0, h * h), g4 = rel_gap(h, mc->step_max, mc->step_max);
            if (g2 < mg) mg = g2;
            if (g3 < mg) mg = g3;
            if (g4 < mg) mg = g4;
        }
        if (t - y > 0.0) {
            double g = mc->k * dd / (t - y);
            if (margin) {
                double sc = fmax(fabs(g), fabs(res));
                double g5 = sc > 0.0 ? rel_gap(g, res, sc) : 0.0;
                if (g5 < mg) mg = g5;
            }
            if (g < res) { res = g; am = i; }
        }
        ph = h;
        t += h < mc->step_max ? h : mc->step_max;
    }
    *nstep = i;
    *argmin = am;
    if (margin) *margin = mg;
    if (res < 0.0) res = 0.0;
    if (res > 1.0) res = 1.0;
    return res;
}

static void normalise3(const double* v, double* L)
{
    double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int a = 0; a < 3; a++) L[a] = v[a] / nv;
}

/* vis[i] for npix shading points (pos/nrm fp32 [npix*3]); light_v need not
 * be unit length (it is normalised).  eps, step_max in world units. */
EXPORT void orc_shadow(const float* sdf, int n, const double* bmin, double extent,
                       const float* pos, const float* nrm, int64_t npix, const double* light_v,
                       double k, int steps, double step_max, double eps, double* vis,
                       int32_t* info /* [npix*3] nstep, argmin, term; may be NULL */,
                       const double* shift /* [npix] origin jitter toward L; may be NULL */)
{
    march_cfg mc = {n, extent / n, extent, eps, k, step_max, steps, bmin};
    double L[3];
    normalise3(light_v, L);
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < npix; i++) {
        double p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        double nn[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
        int ns, am, term;
        vis[i] = march_one(sdf, &mc, p, nn, L, shift ? shift[i] : 0.0, NULL, NULL, &ns, &am, &term, NULL);
        if (info) { info[3 * i] = ns; info[3 * i + 1] = am; info[3 * i + 2] = term; }
    }
}

/* The thin-surface fallback of Sec. 3: where the march steps through a
 * surface thinner than its epsilon, the umbra gets holes; the paper proposes
 * shadow mapping in those regions.  Read here as an exact occlusion test
 * toward the (directional) light from the march's own origin: blocked[i] = 1
 * iff some triangle meets the ray o + t L, t >= 0, with
 * o = fmaf(nrm, 2 eps, pos) in fp32 (the march's origin, single rounding),
 * L the fp32 unit light direction, and the fp32 ray/triangle test of the
 * tracer.  The shadow is then min(vis, 1 - blocked). */
EXPORT void orc_shadow_exact(const float* verts, const int32_t* tris, int64_t nt, const float* pos,
                             const float* nrm, int64_t npix, const float* L, float two_eps, int32_t* blocked)
{
    float* tv0 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te1 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    float* te2 = (float*)malloc(sizeof(float) * 3 * (size_t)(nt > 0 ? nt : 1));
    tri_edges(verts, tris, nt, tv0, te1, te2);
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < npix; i++) {
        float o[3];
        for (int a = 0; a < 3; a++) o[a] = fmaf(nrm[3 * i + a], two_eps, pos[3 * i + a]);
        float t;
        int f;
        blocked[i] = closest_hit(o, L, tv0, te1, te2, nt, &t, &f) >= 0;
    }
    free(tv0); free(te1); free(te2);
}

/* Sec. 2.3 jitters each shadow ray's origin toward the light.  The fraction
 * xi in [0, 1) of pixel i in frame `frame` is the top 24 bits of the first
 * word of Philox-4x32-10 (Salmon et al., SC'11) with counter
 * (i mod 2^32, i div 2^32, frame, 0x53484457 "SHDW") and key (seed lo, seed
 * hi), times 2^-24 (exact in fp32 and fp64). */
EXPORT void orc_shadow_jitter(uint64_t seed, uint32_t frame, int64_t npix, double* xi)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < npix; i++) {
        const uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), frame, 0x53484457u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        xi[i] = (double)(w[0] >> 8) * 0x1p-24;
    }
}

/* ======================================================================
 * Reverse-mode derivative of the Sec. 2.3 march (fp64).
 * Given dvis = dLoss/dvis per point: accumulates dLoss/dsdf (grid) and
 * dLoss/dlight_v (3).  The march is re-run to recover (t_i, h_i); the
 * visibility equals the penumbra term g at its arg-min step i* (first step
 * on ties), so the sweep runs from i* back to 0:
 *   g = k dd / (t - y), y = h^2/(2 ph), dd = sqrt(h^2 - y^2)
 *   h_i = S(o + t_i L),  t_{i+1} = t_i + min(h_i, step_max)
 * Zero derivative where the march stopped on h < eps, where no step set
 * res (res = 1), or where dd was clamped to 0.  L = v/|v|.
 * ====================================================================== */
/* Per shading point, the march's decision margin (see march_one): points
 * whose margin is small may take another discrete path (another step
 * count, another minimising step, termination) when the march is
 * evaluated at another precision. */
EXPORT void orc_shadow_margin(const float* sdf, int n, const double* bmin, double extent,
                              const float* pos, const float* nrm, int64_t npix, const double* light_v,
                              double k, int steps, double step_max, double eps, double* margin)
{
    march_cfg mc = {n, extent / n, extent, eps, k, step_max, steps, bmin};
    double L[3];
    normalise3(light_v, L);
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < npix; i++) {
        double p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        double nn[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
        int ns, am, term;
        march_one(sdf, &mc, p, nn, L, 0.0, NULL, NULL, &ns, &am, &term, &margin[i]);
    }
}

EXPORT void orc_shadow_grad(const float* sdf, int n, const double* bmin, double extent,
                            const float* pos, const float* nrm, int64_t npix, const double* light_v,
                            double k, int steps, double step_max, double eps, const double* dvis,
                            double* dsdf, double* dlight_v)
{
    march_cfg mc = {n, extent / n, extent, eps, k, step_max, steps, bmin};
    double L[3];
    normalise3(light_v, L);
    double gL[3] = {0, 0, 0};
    #pragma omp parallel
    {
        double* ts = (double*)malloc(sizeof(double) * (steps > 0 ? steps : 1));
        double* hs = (double*)malloc(sizeof(double) * (steps > 0 ? steps : 1));
        double lL[3] = {0, 0, 0};
        #pragma omp for schedule(dynamic, 256)
        for (int64_t pi = 0; pi < npix; pi++) {
            if (dvis[pi] == 0.0) continue;
            double p[3] = {pos[3 * pi], pos[3 * pi + 1], pos[3 * pi + 2]};
            double nn[3] = {nrm[3 * pi], nrm[3 * pi + 1], nrm[3 * pi + 2]};
            int ns, am, term;
            march_one(sdf, &mc, p, nn, L, 0.0, ts, hs, &ns, &am, &term, NULL);
            if (term || am < 0) continue;
            double o[3];
            for (int a = 0; a < 3; a++) o[a] = p[a] + 2.0 * eps * nn[a];
            /* derivative of g at step am */
            int i = am;
            double h = hs[i], t = ts[i];
            double ph = i > 0 ? hs[i - 1] : 1e20;
            double y = h * h / (2.0 * ph);
            double a2 = h * h - y * y;
            if (!(a2 > 0.0)) continue;
            double dd = sqrt(a2), den = t - y;
            double dy_dh = h / ph, dy_dph = -y / ph;
            double ddd_dh = (h - y * dy_dh) / dd, ddd_dph = (-y * dy_dph) / dd;
            double gbar = dvis[pi];
            double hbar = gbar * (k * ddd_dh / den + k * dd * dy_dh / (den * den));
            double phbar = i > 0 ? gbar * (k * ddd_dph / den + k * dd * dy_dph / (den * den)) : 0.0;
            double tbar = gbar * (-k * dd / (den * den));
            for (int j = i; j >= 0; j--) {
                /* h_j = S(o + t_j L) */
                double q[3] = {o[0] + ts[j] * L[0], o[1] + ts[j] * L[1], o[2] + ts[j] * L[2]};
                tri_taps tp;
                trilinear(sdf, n, bmin, mc.h, q, &tp);
                double qbar[3] = {0, 0, 0};
                for (int c = 0; c < 8; c++) {
                    #pragma omp atomic
                    dsdf[tp.idx[c]] += hbar * tp.w[c];
                    double fv = (double)sdf[tp.idx[c]];
                    for (int a = 0; a < 3; a++) qbar[a] += hbar * fv * tp.dw[c][a];
                }
                for (int a = 0; a < 3; a++) {
                    tbar += qbar[a] * L[a];
                    lL[a] += qbar[a] * ts[j];
                }
                if (j == 0) break;
                /* t_j = t_{j-1} + min(h_{j-1}, step_max) */
                double hprev = hs[j - 1];
                hbar = (j - 1 == i - 1) ? phbar : 0.0;
                if (hprev < step_max) hbar += tbar;
            }
        }
        #pragma omp critical
        for (int a = 0; a < 3; a++) gL[a] += lL[a];
        free(ts);
        free(hs);
    }
    /* L = v/|v|: dv = (gL - (gL . L) L) / |v| */
    double nv = sqrt(light_v[0] * light_v[0] + light_v[1] * light_v[1] + light_v[2] * light_v[2]);
    double gl = gL[0] * L[0] + gL[1] * L[1] + gL[2] * L[2];
    for (int a = 0; a < 3; a++) dlight_v[a] += (gL[a] - gl * L[a]) / nv;
}
