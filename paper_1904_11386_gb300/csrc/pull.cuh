// Pull helpers of the row-vectorised bulk kernels (sm_103a): a thread owns four consecutive nodes of an
// x-row and moves them as one vector.  Shared by the fused kernel (lbm_kernels.cu) and the two-kernel bulk
// phase (bulk_split.cu).
#pragma once

#include "scbb_internal.cuh"

namespace scbb {

struct Quad {
    float a[4];
};

// populations of direction i (component base cb = S + c*Q*N) arriving at the four nodes x..x+3 of a row
// edge bit 0: the element at x - 1 is not in the lane below (row start or warp edge) and is loaded directly;
// bit 1: likewise for x + 4 and the lane above.
template <int I, typename T>
__device__ __forceinline__ float4 pull4(const LbmParams& p, const T* __restrict__ cb, unsigned int srow, int x,
                                        int segl, int W, int edge, unsigned int lanes) {
    const T* base = cb + (size_t)I * p.N + srow;
    float4 v = pld4(base + x);
    if (dir_x(I) == 1) {            // source x - 1: {x-1, x, x+1, x+2}
        float pw = __shfl_sync(lanes, v.w, (segl + W - 1) & (W - 1), W);
        if (edge & 1) pw = pld(base + (x == 0 ? p.nx - 1 : x - 1));
        v = make_float4(pw, v.x, v.y, v.z);
    } else if (dir_x(I) == -1) {    // source x + 1: {x+1, x+2, x+3, x+4}
        float nx0 = __shfl_sync(lanes, v.x, (segl + 1) & (W - 1), W);
        if (edge & 2) nx0 = pld(base + (x + 4 == p.nx ? 0 : x + 4));
        v = make_float4(v.y, v.z, v.w, nx0);
    }
    return v;
}

struct Mom4 {
    float ra[4], rb[4], jx[4], jy[4], jz[4];
};

template <int I>
__device__ __forceinline__ void acc_dir(Mom4& m, float4 a, float4 b) {
    const float A[4] = {a.x, a.y, a.z, a.w}, B[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        m.ra[k] += A[k];
        m.rb[k] += B[k];
        const float s = A[k] + B[k];
        if (dir_x(I)) m.jx[k] += dir_x(I) * s;
        if (dir_y(I)) m.jy[k] += dir_y(I) * s;
        if (dir_z(I)) m.jz[k] += dir_z(I) * s;
    }
}

struct PullCtx {
    unsigned int rows[3][3];        // [1 - c_y][1 - c_z] row start index of the source row
};

template <int I, typename T>
__device__ __forceinline__ void pull_dir(const LbmParams& p, const T* __restrict__ S, const PullCtx& pc, int x,
                                         int segl, int W, int edge, Mom4& m) {
    const unsigned int srow = pc.rows[1 - dir_y(I)][1 - dir_z(I)];
    float4 a = pull4<I, T>(p, S, srow, x, segl, W, edge, 0xffffffffu);
    float4 b = pull4<I, T>(p, S + (size_t)Q * p.N, srow, x, segl, W, edge, 0xffffffffu);
    if constexpr (is_dev<T>::value) {                  // deviation storage: add the reference back
        const float ra = dir_w(I) * p.rref[0], rb = dir_w(I) * p.rref[1];
        a = make_float4(a.x + ra, a.y + ra, a.z + ra, a.w + ra);
        b = make_float4(b.x + rb, b.y + rb, b.z + rb, b.w + rb);
    }
    acc_dir<I>(m, a, b);
}

template <int... Is>
struct DirList {};

template <typename T, int I, int... Rest>
__device__ __forceinline__ void pull_all(const LbmParams& p, const T* __restrict__ S, const PullCtx& pc, int x,
                                         int segl, int W, int edge, Mom4& m, DirList<I, Rest...>) {
    pull_dir<I, T>(p, S, pc, x, segl, W, edge, m);
    if constexpr (sizeof...(Rest) > 0) pull_all(p, S, pc, x, segl, W, edge, m, DirList<Rest...>{});
}

using AllDirs = DirList<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18>;

__device__ __forceinline__ PullCtx pull_ctx(const LbmParams& p, const int ry[3], int z) {
    int zm = z - 1, zp = z + 1;
    if (!p.walls) {
        zm = zm < 0 ? zm + p.nz : zm;
        zp = zp >= p.nz ? zp - p.nz : zp;
    }
    const unsigned int pz[3] = {(unsigned)zm * p.nxy, (unsigned)z * p.nxy, (unsigned)zp * p.nxy};
    PullCtx pc;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) pc.rows[a][b] = (unsigned)ry[a] + pz[b];
    return pc;
}

template <int I, typename T>
__device__ __forceinline__ float4 pull_comp(const LbmParams& p, const T* __restrict__ cb, const PullCtx& pc, int x,
                                            int segl, int W, int edge, unsigned int lanes) {
    return pull4<I, T>(p, cb, pc.rows[1 - dir_y(I)][1 - dir_z(I)], x, segl, W, edge, lanes);
}

// six psi values x-1 .. x+4 of one ring row (periodic in x)
__device__ __forceinline__ void window6(const float* row, int x, int nx, float w[6]) {
    const float4 v = *reinterpret_cast<const float4*>(row + x);
    w[0] = row[x == 0 ? nx - 1 : x - 1];
    w[1] = v.x; w[2] = v.y; w[3] = v.z; w[4] = v.w;
    w[5] = row[x + 4 == nx ? 0 : x + 4];
}

// Virtual densities of the four wall nodes (x .. x+3, yy) of wall plane z (neutral wetting of the walls):
// the mean of the densities of the five nodes (x', yy, za), (x' +- 1, yy, za), (x', yy +- 1, za) of the
// adjacent fluid plane za, summed in that order.
__device__ __forceinline__ float4 wall_ghost4(const LbmParams& p, const float* __restrict__ a, int x, int yy,
                                              int za) {
    const float* row = a + (size_t)za * p.nxy + yy * p.nx;
    const float* rm = a + (size_t)za * p.nxy + (yy == 0 ? p.ny - 1 : yy - 1) * p.nx;
    const float* rp = a + (size_t)za * p.nxy + (yy == p.ny - 1 ? 0 : yy + 1) * p.nx;
    const float4 c = *reinterpret_cast<const float4*>(row + x);
    const float4 m = *reinterpret_cast<const float4*>(rm + x);
    const float4 pl = *reinterpret_cast<const float4*>(rp + x);
    const float left = row[x == 0 ? p.nx - 1 : x - 1], right = row[x + 4 == p.nx ? 0 : x + 4];
    float4 g;
    g.x = (c.x + left + c.y + m.x + pl.x) * 0.2f;
    g.y = (c.y + c.x + c.z + m.y + pl.y) * 0.2f;
    g.z = (c.z + c.y + c.w + m.z + pl.z) * 0.2f;
    g.w = (c.w + c.z + right + m.w + pl.w) * 0.2f;
    return g;
}

// c_i . v for direction I with only the nonzero terms (a product by a zero component is not folded away
// under IEEE rules)
template <int I>
__device__ __forceinline__ float cdot(float vx, float vy, float vz) {
    float r = 0.f;
    bool first = true;
    auto add = [&](int c, float v) {
        if (c == 0) return;
        const float t = c > 0 ? v : -v;
        r = first ? t : r + t;
        first = false;
    };
    add(dir_x(I), vx);
    add(dir_y(I), vy);
    add(dir_z(I), vz);
    return r;
}

}  // namespace scbb
