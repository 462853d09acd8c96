// Bulk phase in two kernels for tau = 1 (the paper's value): stream + moments, then force + collide.  sm_103a.
//
// With tau = 1 the BGK update (Eq. 1) gives f* = f_eq(rho^c, u_eq^c) exactly, so the collision of a node needs
// nothing of its populations beyond the five moments rho^A, rho^B, j.  Kernel A pulls every node's populations
// once (the stream, Eq. 4) and writes those moments; it has no halo and no barrier, so it is a plain streaming
// read at full occupancy.  Kernel B reads the moments and stages psi of its tile's y-halo rows and z-halo
// planes from the density field (8 bytes per node, L2 hits) instead of pulling 152 bytes of populations for
// them, forms the Shan-Chen force (Eq. 13) and writes f_eq (Eq. 2) of every node.  The moments make one round
// trip through L2 (20 bytes per node).  Quad forms (four nodes per thread, 16-byte vectors) serve nx a multiple
// of 4, scalar forms (one node per thread) any nx.
//
// Batches: one cooperative launch runs kernel A over every box, waits at a grid barrier that gives up after a
// spin limit (device error bit 4, SCBB_E_TIMEOUT), and runs kernel B over every box's (tile, z-segment) items.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "async_copy.cuh"
#include "pull.cuh"
#include "pdl.cuh"
#include "scbb_internal.cuh"

namespace scbb {

// Kernel A: one thread per four consecutive nodes of a row (float4 loads; the x-shifts of the pull are warp
// shuffles, see pull4), every fluid node of the lattice once.  Writes rho^c to rho[c][n] and j to J[d][n],
// summed over the directions in the same order as the fused kernel, so both give the same bits.
// Moments of one node (x, y, z): pulled populations (reconstructed at on-site velocity planes), summed over the
// directions in the same order as the quad form.
template <typename T>
__device__ __forceinline__ void node_moments(const LbmParams& p, const T* __restrict__ S, float* __restrict__ rho,
                                             float* __restrict__ J, int x, int y, int z) {
    Cols k;
    k.cx[0] = x == 0 ? p.nx - 1 : x - 1; k.cx[1] = x; k.cx[2] = x == p.nx - 1 ? 0 : x + 1;
    k.ry[0] = (y == 0 ? p.ny - 1 : y - 1) * p.nx; k.ry[1] = y * p.nx; k.ry[2] = (y == p.ny - 1 ? 0 : y + 1) * p.nx;
    float f[2 * Q];
    pull(p, S, k, z, f);
    if (is_onsite_plane(p, z)) onsite_fix(p, z, f);
    float ra = 0.f, rb = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        ra += f[i];
        rb += f[Q + i];
        const float s = f[i] + f[Q + i];
        if (dir_x(i)) jx += dir_x(i) * s;
        if (dir_y(i)) jy += dir_y(i) * s;
        if (dir_z(i)) jz += dir_z(i) * s;
    }
    const unsigned int n = (unsigned)x + (unsigned)k.ry[1] + (unsigned)z * p.nxy;
    rho[n] = ra;
    rho[p.N + n] = rb;
    J[n] = jx;
    J[p.N + n] = jy;
    J[2 * (size_t)p.N + n] = jz;
}

template <typename T>
__device__ __forceinline__ void moments4_quad(const LbmParams& p, const T* __restrict__ S, float* __restrict__ rho,
                                              float* __restrict__ J, unsigned int g0, unsigned int total) {
    const int NQ = p.nx >> 2;
    const bool live = g0 < total;
    const unsigned int g = live ? g0 : total - 1;       // the tail of the last warp shadows the last quad
    const unsigned int row = g / (unsigned)NQ;
    const int q = (int)(g - row * (unsigned)NQ);
    const int y = (int)(row % (unsigned)p.ny);
    const int z = p.zf0 + (int)(row / (unsigned)p.ny);
    const int x = 4 * q;
    const int lane = threadIdx.x & 31;
    // rows of a power-of-two number of quads up to 32 fill whole lane segments (their shuffle wrap is the
    // periodic boundary); any other row shuffles across the warp and loads the element beyond a warp edge or
    // the periodic wrap directly.  Live rows are whole, so a live lane's shuffle partner is live or loads.
    const bool seg_rows = NQ <= 32 && (NQ & (NQ - 1)) == 0;
    const int W = seg_rows ? NQ : 32;
    const int segl = seg_rows ? (q & (W - 1)) : lane;
    const int edge = seg_rows ? 0 : (((q == 0 || lane == 0) ? 1 : 0) | ((q == NQ - 1 || lane == 31) ? 2 : 0));
    const int ry[3] = {(y == 0 ? p.ny - 1 : y - 1) * p.nx, y * p.nx, (y == p.ny - 1 ? 0 : y + 1) * p.nx};
    if (p.onsite && __any_sync(0xffffffffu, is_onsite_plane(p, z))) {
        // a warp touching an on-site velocity plane takes its nodes one at a time (the boundary's reconstruction
        // needs the populations themselves; the vote keeps the branch uniform, and there are no shuffles in it)
        if (!live) return;
#pragma unroll 1
        for (int k = 0; k < 4; k++) node_moments<T>(p, S, rho, J, x + k, y, z);
        return;
    }
    Mom4 m;
#pragma unroll
    for (int k = 0; k < 4; k++) m.ra[k] = m.rb[k] = m.jx[k] = m.jy[k] = m.jz[k] = 0.f;
    const PullCtx pc = pull_ctx(p, ry, z);
    pull_all(p, S, pc, x, segl, W, edge, m, AllDirs{});
    if (!live) return;
    const unsigned int n0 = (unsigned)x + (unsigned)ry[1] + (unsigned)z * p.nxy;
    *reinterpret_cast<float4*>(rho + n0) = make_float4(m.ra[0], m.ra[1], m.ra[2], m.ra[3]);
    *reinterpret_cast<float4*>(rho + p.N + n0) = make_float4(m.rb[0], m.rb[1], m.rb[2], m.rb[3]);
    *reinterpret_cast<float4*>(J + n0) = make_float4(m.jx[0], m.jx[1], m.jx[2], m.jx[3]);
    *reinterpret_cast<float4*>(J + p.N + n0) = make_float4(m.jy[0], m.jy[1], m.jy[2], m.jy[3]);
    *reinterpret_cast<float4*>(J + 2 * (size_t)p.N + n0) = make_float4(m.jz[0], m.jz[1], m.jz[2], m.jz[3]);
}

// Kernel A, one node per thread (any nx): the same moments, summed in the same order as the quad form.
template <typename T>
__device__ __forceinline__ void moments1_node(const LbmParams& p, const T* __restrict__ S, float* __restrict__ rho,
                                              float* __restrict__ J, unsigned int g, unsigned int total) {
    if (g >= total) return;
    const unsigned int row = g / (unsigned)p.nx;
    const int x = (int)(g - row * (unsigned)p.nx);
    node_moments<T>(p, S, rho, J, x, (int)(row % (unsigned)p.ny), p.zf0 + (int)(row / (unsigned)p.ny));
}

// Virtual density of the wall node (x, yy) of a wall plane whose adjacent fluid plane is za (neutral
// wetting): the mean over (x, yy, za), (x -+ 1, yy, za), (x, yy -+ 1, za), summed in the order of the quad form.
__device__ __forceinline__ float wall_ghost1(const LbmParams& p, const float* __restrict__ a, int x, int yy, int za) {
    const float* row = a + (size_t)za * p.nxy + yy * p.nx;
    const float* rm = a + (size_t)za * p.nxy + (yy == 0 ? p.ny - 1 : yy - 1) * p.nx;
    const float* rp = a + (size_t)za * p.nxy + (yy == p.ny - 1 ? 0 : yy + 1) * p.nx;
    return (row[x] + row[x == 0 ? p.nx - 1 : x - 1] + row[x == p.nx - 1 ? 0 : x + 1] + rm[x] + rp[x]) * 0.2f;
}

// Kernel B, one node per thread (any nx): one work item is TY whole rows (tile `tile`) marching through z-segment
// `seg` of `nseg`, the block's threads covering the TY rows node by node (at least 2 nx threads, for the halo
// rows); the arithmetic is the quad form's for one node.
template <int MODE, typename T>
__device__ __forceinline__ void collide1_tile(const LbmParams& p, T* __restrict__ D, const float* __restrict__ rho,
                                              const float* __restrict__ J, float* __restrict__ ghost,
                                              const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
                                              float* __restrict__ u_out, int* __restrict__ err, int TY, int tile,
                                              int seg, int nseg, float* ring) {
    constexpr bool IBM = MODE == 1;
    const int nx = p.nx;
    const int RR = TY + 2;
    const int t = threadIdx.x;
    const int nreal = nx * TY;
    const int tr = t < nreal ? t : nreal - 1;
    const int r = tr / nx + 1;
    const int x = tr - (r - 1) * nx;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int y0 = tile * TY;
    const int gy = y0 + r - 1;
    const bool active = t < nreal && gy < p.ny;
    const int plane_sz = RR * nx;
    const int ry[3] = {(gy == 0 ? p.ny - 1 : gy - 1) * nx, gy * nx, (gy + 1 >= p.ny ? 0 : gy + 1) * nx};

    const int nzf = p.zf1 - p.zf0;
    const int zs = p.zf0 + (int)(((long long)seg * nzf) / nseg);
    const int ze = p.zf0 + (int)(((long long)(seg + 1) * nzf) / nseg);
    if (zs >= ze) return;
    const int dz = (seg & 1) ? 1 : -1;
    const int z_first = dz > 0 ? zs : ze - 1;
    const int L = ze - zs;
    auto zwrap = [&](int z) { return p.walls ? z : (z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z)); };

    const bool own_q = t < nreal;
    const bool halo_q = t < 2 * nx;
    const int hr = t < nx ? 0 : TY + 1;
    const int hx = t < nx ? t : t - nx;
    int hy = hr == 0 ? y0 - 1 : y0 + TY;
    hy = hy < 0 ? hy + p.ny : (hy >= p.ny ? hy - p.ny : hy);
    const int gyw = gy >= p.ny ? gy - p.ny : gy;
    auto load_n = [&](int z, int xq, int yq, float& a, float& b) {
        if (is_wall_plane(p, z)) {
            const int za = z == 0 ? 1 : p.nz - 2;
            a = wall_ghost1(p, rho, xq, yq, za);
            b = wall_ghost1(p, rho + p.N, xq, yq, za);
        } else {
            const size_t n = (size_t)z * p.nxy + yq * nx + xq;
            a = rho[n];
            b = rho[p.N + n];
        }
    };
    auto store = [&](int z, int slot, float a, float b) {
        float* base = ring + (size_t)slot * 2 * plane_sz;
        if (own_q) {
            base[r * nx + x] = psi_fn(a, p.psi_kind);
            base[plane_sz + r * nx + x] = psi_fn(b, p.psi_kind);
            if (active && is_wall_plane(p, z)) {
                const int w = z == 0 ? 0 : 1;
                ghost[(w * 2 + 0) * p.nxy + gy * nx + x] = a;
                ghost[(w * 2 + 1) * p.nxy + gy * nx + x] = b;
            }
        }
        if (halo_q) {
            float ha, hb;
            load_n(z, hx, hy, ha, hb);
            base[hr * nx + hx] = psi_fn(ha, p.psi_kind);
            base[plane_sz + hr * nx + hx] = psi_fn(hb, p.psi_kind);
        }
    };

    float ra = 0.f, rb = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
    {
        const int zb = zwrap(z_first - dz);
        float a = 0.f, b = 0.f;
        if (own_q) load_n(zb, x, gyw, a, b);
        store(zb, 0, a, b);
        if (own_q) load_n(z_first, x, gyw, ra, rb);
        store(z_first, 1, ra, rb);
    }
    float an = 0.f, bn = 0.f;                            // densities of plane z + 1 (loaded a plane ahead)
    if (own_q) load_n(zwrap(z_first + dz), x, gyw, an, bn);

    for (int rel = 0; rel < L; rel++) {
        const int z = z_first + rel * dz;
        store(zwrap(z + dz), (rel + 2) & 3, an, bn);
        const float a1 = an, b1 = bn;
        if (rel + 1 < L && own_q) load_n(zwrap(z + 2 * dz), x, gyw, an, bn);
        const unsigned int n0 = (unsigned)x + (unsigned)ry[1] + (unsigned)z * p.nxy;
        if (active) {
            jx = J[n0];
            jy = J[p.N + n0];
            jz = J[2 * (size_t)p.N + n0];
        }
        __syncthreads();
        if (active) {
            // ---- Shan-Chen force (Eq. 13) from the psi ring, the quad form's sums for one node
            const int s_back = rel & 3, s_ahead = (rel + 2) & 3;
            const float* pm = ring + (size_t)(dz > 0 ? s_back : s_ahead) * 2 * plane_sz;
            const float* p0 = ring + (size_t)((rel + 1) & 3) * 2 * plane_sz;
            const float* pp = ring + (size_t)(dz > 0 ? s_ahead : s_back) * 2 * plane_sz;
            float S[2][3], ps[2];
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const int co = c * plane_sz;
                const float* c00 = p0 + co + r * nx;
                const float* cyp = p0 + co + (r + 1) * nx;
                const float* cym = p0 + co + (r - 1) * nx;
                const float* czp = pp + co + r * nx;
                const float* czm = pm + co + r * nx;
                const float Cpp = pp[co + (r + 1) * nx + x], Cmp = pp[co + (r - 1) * nx + x];
                const float Cpm = pm[co + (r + 1) * nx + x], Cmm = pm[co + (r - 1) * nx + x];
                S[c][0] = (c00[xp] - c00[xm]) * (1.f / 18.f) +
                          ((cyp[xp] - cyp[xm]) + (cym[xp] - cym[xm]) + (czp[xp] - czp[xm]) + (czm[xp] - czm[xm])) *
                              (1.f / 36.f);
                const float ty = (cyp[xp] + cyp[xm]) - (cym[xp] + cym[xm]);
                const float tz = (czp[xp] + czp[xm]) - (czm[xp] + czm[xm]);
                S[c][1] = (cyp[x] - cym[x]) * (1.f / 18.f) + (ty + ((Cpp + Cpm) - (Cmp + Cmm))) * (1.f / 36.f);
                S[c][2] = (czp[x] - czm[x]) * (1.f / 18.f) + (tz + ((Cpp + Cmp) - (Cpm + Cmm))) * (1.f / 36.f);
                ps[c] = c00[x];
            }
            const float rt = ra + rb;
            const float irt = 1.f / rt;
            float FA[3], FB[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                FA[d] = -ps[0] * p.G * S[1][d] + ra * p.g[d];
                FB[d] = -ps[1] * p.G * S[0][d] + rb * p.g[d];
            }
            const bool ibm_node = IBM && ((__ldg(mask + (n0 >> 5)) >> (n0 & 31)) & 1u);
            if (ibm_node) {
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const float fi = ibm_unfix(Fibm[(size_t)d * p.N + n0]);
                    FA[d] += ra * irt * fi;
                    FB[d] += rb * irt * fi;
                }
            }
            const float ux = jx * irt, uy = jy * irt, uz = jz * irt;
            if (!(rt > 0.f) || !(ux * ux + uy * uy + uz * uz <= 0.09f)) atomicOr(err, 1);
            const float ta = ra > 0.f ? p.tau / ra : 0.f, tb = rb > 0.f ? p.tau / rb : 0.f;
            const float uA0 = ux + ta * FA[0], uA1 = uy + ta * FA[1], uA2 = uz + ta * FA[2];
            const float uB0 = ux + tb * FB[0], uB1 = uy + tb * FB[1], uB2 = uz + tb * FB[2];
            const float aA = 1.f - 1.5f * (uA0 * uA0 + uA1 * uA1 + uA2 * uA2);
            const float aB = 1.f - 1.5f * (uB0 * uB0 + uB1 * uB1 + uB2 * uB2);
            const float vA[3] = {3.f * uA0, 3.f * uA1, 3.f * uA2}, vB[3] = {3.f * uB0, 3.f * uB1, 3.f * uB2};
            if (ibm_node) {
                u_out[n0] = (jx + 0.5f * (FA[0] + FB[0])) * irt;
                u_out[(size_t)p.N + n0] = (jy + 0.5f * (FA[1] + FB[1])) * irt;
                u_out[(size_t)2 * p.N + n0] = (jz + 0.5f * (FA[2] + FB[2])) * irt;
            }
            // ---- equilibrium (Eq. 2) = the post-collision populations, by opposite-direction pairs
            const bool wall_next = p.walls && (z == 1 || z == p.nz - 2);
            float sA = 0.f, sB = 0.f;
            auto store_dir = [&](auto Ic, float oA, float oB) {
                constexpr int I = decltype(Ic)::value;
                if (dir_z(I) != 0 && wall_next && is_wall_plane(p, z + dir_z(I))) {
                    // half-way bounce-back on a moving wall (Eq. 11), stored where the node pulls opp(I) from
                    const float* U = (z + dir_z(I) == 0) ? p.ulo : p.uhi;
                    const float cU = 6.f * dir_w(I) * (dir_x(I) * U[0] + dir_y(I) * U[1] + dir_z(I) * U[2]);
                    int xd = x + dir_x(I);
                    xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
                    const unsigned int dn = (unsigned)ry[1 + dir_y(I)] + (unsigned)(z + dir_z(I)) * p.nxy + xd;
                    pst(D + (size_t)dir_opp(I) * p.N + dn, oA - cU * ra);
                    pst(D + (size_t)(Q + dir_opp(I)) * p.N + dn, oB - cU * rb);
                } else {
                    pst(D + (size_t)I * p.N + n0, oA);
                    pst(D + (size_t)(Q + I) * p.N + n0, oB);
                }
            };
            auto emit_pair = [&](auto Ic) {
                constexpr int I = decltype(Ic)::value;
                constexpr float W = dir_w(I);
                const float qA = cdot<I>(vA[0], vA[1], vA[2]), qB = cdot<I>(vB[0], vB[1], vB[2]);
                const float hA = fmaf(0.5f * qA, qA, aA), hB = fmaf(0.5f * qB, qB, aB);
                const float wA = W * ra, wB = W * rb;
                float oA, oB, pA, pB;
                if constexpr (is_dev<T>::value) {      // deviations from W rref^c
                    const float dA = W * p.rref[0], dB = W * p.rref[1];
                    oA = pround(wA * (hA + qA) - dA, D); oB = pround(wB * (hB + qB) - dB, D);
                    pA = pround(wA * (hA - qA) - dA, D); pB = pround(wB * (hB - qB) - dB, D);
                } else {
                    oA = pround(wA * (hA + qA), D); oB = pround(wB * (hB + qB), D);
                    pA = pround(wA * (hA - qA), D); pB = pround(wB * (hB - qB), D);
                }
                sA += oA + pA;
                sB += oB + pB;
                store_dir(std::integral_constant<int, I>{}, oA, oB);
                store_dir(std::integral_constant<int, I + 1>{}, pA, pB);
            };
            emit_pair(std::integral_constant<int, 1>{});  emit_pair(std::integral_constant<int, 3>{});
            emit_pair(std::integral_constant<int, 5>{});  emit_pair(std::integral_constant<int, 7>{});
            emit_pair(std::integral_constant<int, 9>{});  emit_pair(std::integral_constant<int, 11>{});
            emit_pair(std::integral_constant<int, 13>{}); emit_pair(std::integral_constant<int, 15>{});
            emit_pair(std::integral_constant<int, 17>{});
            float oA = (ra - dev_ref<T>(p, 0)) - sA, oB = (rb - dev_ref<T>(p, 1)) - sB;
            if (sizeof(T) == 2) {           // unbiased rounding of the mass-closing value
                const uint32_t h = dither_bits(n0, ra, rb);
                oA = pdither(oA, h >> 16, D);
                oB = pdither(oB, h & 0xffffu, D);
            }
            store_dir(std::integral_constant<int, 0>{}, oA, oB);
        }
        ra = a1;
        rb = b1;
    }
}

// Collision of the four nodes x .. x+3 of ring row r (global row offsets ry) in plane z, the rel-th plane of its
// z-segment marching in direction dz: the Shan-Chen force (Eq. 13) from the psi ring (planes z - 1 .. z + 1 in
// the slots that rel and dz select), the equilibrium velocities and the f_eq stores (Eq. 2, with the moving-wall
// bounce-back of Eq. 11 next to a wall).  a4, b4: the nodes' densities; jx4, jy4, jz4: their momentum.
template <int MODE, typename T>
__device__ __forceinline__ void collide4_plane(const LbmParams& p, T* __restrict__ D, const float* ring, int plane_sz,
                                               int rel, int dz, int r, int x, const int ry[3], int z, float4 a4,
                                               float4 b4, float4 jx4, float4 jy4, float4 jz4,
                                               const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
                                               float* __restrict__ u_out, int* __restrict__ err) {
    constexpr bool IBM = MODE == 1;
    const int nx = p.nx;
    const unsigned int n0 = (unsigned)x + (unsigned)ry[1] + (unsigned)z * p.nxy;
    // ---- Shan-Chen force (Eq. 13) for the four nodes from the psi ring.  Per component, with the ring
    // rows R = (c_y, c_z) of the planes z - 1 .. z + 1: S_x = (1/18) D(0,0) + (1/36) sum of D over the four
    // edge rows, D = psi(x+1) - psi(x-1); S_y and S_z from the centre values C and the x-pair sums T of the
    // rows above and below (weights 1/18 for the axis rows, 1/36 for the edge and corner rows)
    const int s_back = rel & 3, s_ahead = (rel + 2) & 3;
    const float* pm = ring + (size_t)(dz > 0 ? s_back : s_ahead) * 2 * plane_sz;   // plane z - 1
    const float* p0 = ring + (size_t)((rel + 1) & 3) * 2 * plane_sz;               // plane z
    const float* pp = ring + (size_t)(dz > 0 ? s_ahead : s_back) * 2 * plane_sz;   // plane z + 1
    float SA[3][4], SB[3][4], psA[4], psB[4];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int co = c * plane_sz;
        float w00[6], wyp[6], wym[6], wzp[6], wzm[6];
        window6(p0 + co + r * nx, x, nx, w00);
        window6(p0 + co + (r + 1) * nx, x, nx, wyp);
        window6(p0 + co + (r - 1) * nx, x, nx, wym);
        window6(pp + co + r * nx, x, nx, wzp);
        window6(pm + co + r * nx, x, nx, wzm);
        const float4 cpp = *reinterpret_cast<const float4*>(pp + co + (r + 1) * nx + x);   // (+y, +z)
        const float4 cmp = *reinterpret_cast<const float4*>(pp + co + (r - 1) * nx + x);   // (-y, +z)
        const float4 cpm = *reinterpret_cast<const float4*>(pm + co + (r + 1) * nx + x);   // (+y, -z)
        const float4 cmm = *reinterpret_cast<const float4*>(pm + co + (r - 1) * nx + x);   // (-y, -z)
        const float Cpp[4] = {cpp.x, cpp.y, cpp.z, cpp.w}, Cmp[4] = {cmp.x, cmp.y, cmp.z, cmp.w};
        const float Cpm[4] = {cpm.x, cpm.y, cpm.z, cpm.w}, Cmm[4] = {cmm.x, cmm.y, cmm.z, cmm.w};
        float(&S)[3][4] = c == 0 ? SA : SB;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float dx = (w00[k + 2] - w00[k]) * (1.f / 18.f) +
                             ((wyp[k + 2] - wyp[k]) + (wym[k + 2] - wym[k]) + (wzp[k + 2] - wzp[k]) +
                              (wzm[k + 2] - wzm[k])) * (1.f / 36.f);
            const float ty = (wyp[k + 2] + wyp[k]) - (wym[k + 2] + wym[k]);
            const float tz = (wzp[k + 2] + wzp[k]) - (wzm[k + 2] + wzm[k]);
            const float dy = (wyp[k + 1] - wym[k + 1]) * (1.f / 18.f) +
                             (ty + ((Cpp[k] + Cpm[k]) - (Cmp[k] + Cmm[k]))) * (1.f / 36.f);
            const float dzv = (wzp[k + 1] - wzm[k + 1]) * (1.f / 18.f) +
                              (tz + ((Cpp[k] + Cmp[k]) - (Cpm[k] + Cmm[k]))) * (1.f / 36.f);
            S[0][k] = dx; S[1][k] = dy; S[2][k] = dzv;
            if (c == 0) psA[k] = w00[k + 1]; else psB[k] = w00[k + 1];
        }
    }

    uint32_t bits = 0;
    if (IBM) bits = (__ldg(mask + (n0 >> 5)) >> (n0 & 31)) & 0xFu;
    const float ra[4] = {a4.x, a4.y, a4.z, a4.w}, rb[4] = {b4.x, b4.y, b4.z, b4.w};
    const float jxa[4] = {jx4.x, jx4.y, jx4.z, jx4.w}, jya[4] = {jy4.x, jy4.y, jy4.z, jy4.w},
                jza[4] = {jz4.x, jz4.y, jz4.z, jz4.w};
    // per node and component: 3 u_eq (the c_i . u of Eq. 2 scaled by 1/cs^2 = 3), a = 1 - 1.5 u.u, and the
    // weighted densities w rho for the axis (1/18) and diagonal (1/36) directions
    float vA[4][3], vB[4][3], aA[4], aB[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float rt = ra[k] + rb[k];
        const float irt = 1.f / rt;
        float FA[3], FB[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            FA[d] = -psA[k] * p.G * SB[d][k] + ra[k] * p.g[d];
            FB[d] = -psB[k] * p.G * SA[d][k] + rb[k] * p.g[d];
        }
        if (IBM && ((bits >> k) & 1u)) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const float fi = ibm_unfix(Fibm[(size_t)d * p.N + n0 + k]);
                FA[d] += ra[k] * irt * fi;
                FB[d] += rb[k] * irt * fi;
            }
        }
        const float ux = jxa[k] * irt, uy = jya[k] * irt, uz = jza[k] * irt;
        if (!(rt > 0.f) || !(ux * ux + uy * uy + uz * uz <= 0.09f)) atomicOr(err, 1);
        const float ta = ra[k] > 0.f ? p.tau / ra[k] : 0.f, tb = rb[k] > 0.f ? p.tau / rb[k] : 0.f;
        const float uA0 = ux + ta * FA[0], uA1 = uy + ta * FA[1], uA2 = uz + ta * FA[2];
        const float uB0 = ux + tb * FB[0], uB1 = uy + tb * FB[1], uB2 = uz + tb * FB[2];
        aA[k] = 1.f - 1.5f * (uA0 * uA0 + uA1 * uA1 + uA2 * uA2);
        aB[k] = 1.f - 1.5f * (uB0 * uB0 + uB1 * uB1 + uB2 * uB2);
        vA[k][0] = 3.f * uA0; vA[k][1] = 3.f * uA1; vA[k][2] = 3.f * uA2;
        vB[k][0] = 3.f * uB0; vB[k][1] = 3.f * uB1; vB[k][2] = 3.f * uB2;
        if (IBM && ((bits >> k) & 1u)) {
            u_out[n0 + k] = (jxa[k] + 0.5f * (FA[0] + FB[0])) * irt;
            u_out[(size_t)p.N + n0 + k] = (jya[k] + 0.5f * (FA[1] + FB[1])) * irt;
            u_out[(size_t)2 * p.N + n0 + k] = (jza[k] + 0.5f * (FA[2] + FB[2])) * irt;
        }
    }
    // ---- equilibrium (Eq. 2) = the post-collision populations.  For a direction pair i, opp(i) with
    // q = 3 c_i.u: f_eq = w rho (a + q + q^2 / 2) and w rho (a - q + q^2 / 2), so the pair shares h = a + q^2/2.
    const bool wall_next = p.walls && (z == 1 || z == p.nz - 2);
    float sA[4], sB[4];
#pragma unroll
    for (int k = 0; k < 4; k++) sA[k] = sB[k] = 0.f;
    auto store_dir = [&](auto Ic, const float (&oA)[4], const float (&oB)[4]) {
        constexpr int I = decltype(Ic)::value;
        if (dir_z(I) != 0 && wall_next && is_wall_plane(p, z + dir_z(I))) {
            // half-way bounce-back on a moving wall (Eq. 11), stored where the node pulls opp(I) from
            const float* U = (z + dir_z(I) == 0) ? p.ulo : p.uhi;
            const float cU = 6.f * dir_w(I) * (dir_x(I) * U[0] + dir_y(I) * U[1] + dir_z(I) * U[2]);
            const unsigned int drow = (unsigned)ry[1 + dir_y(I)] + (unsigned)(z + dir_z(I)) * p.nxy;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                int xd = x + k + dir_x(I);
                xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
                pst(D + (size_t)dir_opp(I) * p.N + drow + xd, oA[k] - cU * ra[k]);
                pst(D + (size_t)(Q + dir_opp(I)) * p.N + drow + xd, oB[k] - cU * rb[k]);
            }
        } else {
            pst4(D + (size_t)I * p.N + n0, make_float4(oA[0], oA[1], oA[2], oA[3]));
            pst4(D + (size_t)(Q + I) * p.N + n0, make_float4(oB[0], oB[1], oB[2], oB[3]));
        }
    };
    auto emit_pair = [&](auto Ic) {
        constexpr int I = decltype(Ic)::value;             // odd: I and I + 1 = opp(I)
        constexpr float W = dir_w(I);
        float oA[4], oB[4], qA4[4], qB4[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float qA = cdot<I>(vA[k][0], vA[k][1], vA[k][2]);
            const float qB = cdot<I>(vB[k][0], vB[k][1], vB[k][2]);
            const float hA = fmaf(0.5f * qA, qA, aA[k]), hB = fmaf(0.5f * qB, qB, aB[k]);
            const float wA = W * ra[k], wB = W * rb[k];
            if constexpr (is_dev<T>::value) {          // deviations from W rref^c
                const float dA = W * p.rref[0], dB = W * p.rref[1];
                oA[k] = pround(wA * (hA + qA) - dA, D);
                oB[k] = pround(wB * (hB + qB) - dB, D);
                qA4[k] = pround(wA * (hA - qA) - dA, D);
                qB4[k] = pround(wB * (hB - qB) - dB, D);
            } else {
                oA[k] = pround(wA * (hA + qA), D);
                oB[k] = pround(wB * (hB + qB), D);
                qA4[k] = pround(wA * (hA - qA), D);
                qB4[k] = pround(wB * (hB - qB), D);
            }
            sA[k] += oA[k] + qA4[k];
            sB[k] += oB[k] + qB4[k];
        }
        store_dir(std::integral_constant<int, I>{}, oA, oB);
        store_dir(std::integral_constant<int, I + 1>{}, qA4, qB4);
    };
    emit_pair(std::integral_constant<int, 1>{});  emit_pair(std::integral_constant<int, 3>{});
    emit_pair(std::integral_constant<int, 5>{});  emit_pair(std::integral_constant<int, 7>{});
    emit_pair(std::integral_constant<int, 9>{});  emit_pair(std::integral_constant<int, 11>{});
    emit_pair(std::integral_constant<int, 13>{}); emit_pair(std::integral_constant<int, 15>{});
    emit_pair(std::integral_constant<int, 17>{});
    {
        // the rest population closes each node's mass over the values as stored
        float oA[4], oB[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            oA[k] = (ra[k] - dev_ref<T>(p, 0)) - sA[k];
            oB[k] = (rb[k] - dev_ref<T>(p, 1)) - sB[k];
            if (sizeof(T) == 2) {       // unbiased rounding of the mass-closing value
                const uint32_t h = dither_bits(n0 + k, ra[k], rb[k]);
                oA[k] = pdither(oA[k], h >> 16, D);
                oB[k] = pdither(oB[k], h & 0xffffu, D);
            }
        }
        store_dir(std::integral_constant<int, 0>{}, oA, oB);
    }
}

// Kernel B, one work item: TY whole rows (tile `tile`) marching through z-segment `seg` of `nseg`; one thread per
// quad of a tile row; the block calls it with all its threads (it synchronises).  psi of the tile rows and the two halo rows, for the planes z - 1 .. z + 1, sits in a
// four-plane shared ring filled from the density field (wall planes: the ghost densities, computed here from
// the adjacent fluid plane and written out for the boundary kernel by the CTA that owns the rows).
template <int MODE, typename T>
__device__ __forceinline__ void collide4_tile(const LbmParams& p, T* __restrict__ D, const float* __restrict__ rho,
                                              const float* __restrict__ J, float* __restrict__ ghost,
                                              const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
                                              float* __restrict__ u_out, int* __restrict__ err, int TY, int tile,
                                              int seg, int nseg, float* ring) {
    constexpr bool IBM = MODE == 1;
    const int nx = p.nx;
    const int NQ = nx >> 2;
    const int RR = TY + 2;
    const int t = threadIdx.x;
    const int nreal = NQ * TY;
    const int tr = t < nreal ? t : nreal - 1;
    const int r = tr / NQ + 1;                           // ring row 1 .. TY (0 and TY + 1 are the halo rows)
    const int q = tr - (r - 1) * NQ;
    const int x = 4 * q;
    const int y0 = tile * TY;
    const int gy = y0 + r - 1;
    const bool active = t < nreal && gy < p.ny;
    const int plane_sz = RR * nx;
    const int ry[3] = {(gy == 0 ? p.ny - 1 : gy - 1) * nx, gy * nx, (gy + 1 >= p.ny ? 0 : gy + 1) * nx};

    const int nzf = p.zf1 - p.zf0;
    const int zs = p.zf0 + (int)(((long long)seg * nzf) / nseg);
    const int ze = p.zf0 + (int)(((long long)(seg + 1) * nzf) / nseg);
    if (zs >= ze) return;
    const int dz = (seg & 1) ? 1 : -1;
    const int z_first = dz > 0 ? zs : ze - 1;
    const int L = ze - zs;
    auto zwrap = [&](int z) { return p.walls ? z : (z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z)); };

    // Ring fill, software-pipelined: thread t fills the quad of its own tile row (t < nreal) and, for t < 2 NQ,
    // one quad of the halo row below (t < NQ) or above.  The densities of plane z + 2 are loaded before plane z's
    // barrier and written into the ring one plane later, so their latency hides behind the collision.  A thread's own densities come from its fill.  Wall planes hold the ghost densities,
    // computed here from the adjacent fluid plane; the CTA that owns the rows writes them out for the boundary
    // kernel.
    struct Fill {
        float4 a, b;
    };
    const bool own_q = t < nreal;
    const bool halo_q = t < 2 * NQ;
    const int hr = t < NQ ? 0 : TY + 1;                  // ring row of the halo quad
    const int hx = 4 * (t < NQ ? t : t - NQ);
    int hy = hr == 0 ? y0 - 1 : y0 + TY;
    hy = hy < 0 ? hy + p.ny : (hy >= p.ny ? hy - p.ny : hy);
    const int gyw = gy >= p.ny ? gy - p.ny : gy;          // rows past ny (last tile) wrap, and are not collided
    // densities (ghost densities on a wall plane) of plane z at the quad (xq, yq)
    auto load_q = [&](int z, int xq, int yq, float4& a, float4& b) {
        if (is_wall_plane(p, z)) {
            const int za = z == 0 ? 1 : p.nz - 2;
            a = wall_ghost4(p, rho, xq, yq, za);
            b = wall_ghost4(p, rho + p.N, xq, yq, za);
        } else {
            const size_t n = (size_t)z * p.nxy + yq * nx + xq;
            a = *reinterpret_cast<const float4*>(rho + n);
            b = *reinterpret_cast<const float4*>(rho + p.N + n);
        }
    };
    auto load = [&](int z) {
        Fill f;
        f.a = f.b = make_float4(0.f, 0.f, 0.f, 0.f);
        if (own_q) load_q(z, x, gyw, f.a, f.b);
        return f;
    };
    auto psi4 = [&](float4 v) {
        return make_float4(psi_fn(v.x, p.psi_kind), psi_fn(v.y, p.psi_kind), psi_fn(v.z, p.psi_kind),
                           psi_fn(v.w, p.psi_kind));
    };
    auto store = [&](int z, int slot, const Fill& f) {
        float* base = ring + (size_t)slot * 2 * plane_sz;
        if (own_q) {
            *reinterpret_cast<float4*>(base + r * nx + x) = psi4(f.a);
            *reinterpret_cast<float4*>(base + plane_sz + r * nx + x) = psi4(f.b);
            if (active && is_wall_plane(p, z)) {
                const int w = z == 0 ? 0 : 1;
                *reinterpret_cast<float4*>(ghost + (w * 2 + 0) * p.nxy + gy * nx + x) = f.a;
                *reinterpret_cast<float4*>(ghost + (w * 2 + 1) * p.nxy + gy * nx + x) = f.b;
            }
        }
        if (halo_q) {
            float4 ha, hb;
            load_q(z, hx, hy, ha, hb);
            *reinterpret_cast<float4*>(base + hr * nx + hx) = psi4(ha);
            *reinterpret_cast<float4*>(base + plane_sz + hr * nx + hx) = psi4(hb);
        }
    };
    auto load_j = [&](int z, float4& jx, float4& jy, float4& jz) {
        const size_t n = (size_t)x + (size_t)ry[1] + (size_t)z * p.nxy;
        jx = *reinterpret_cast<const float4*>(J + n);
        jy = *reinterpret_cast<const float4*>(J + p.N + n);
        jz = *reinterpret_cast<const float4*>(J + 2 * (size_t)p.N + n);
    };

    float4 a4, b4, jx4, jy4, jz4;                        // densities and momentum of the plane being collided
    jx4 = jy4 = jz4 = make_float4(0.f, 0.f, 0.f, 0.f);
    {
        const int zb = zwrap(z_first - dz);
        store(zb, 0, load(zb));
        const Fill f1 = load(z_first);
        store(z_first, 1, f1);
        a4 = f1.a;
        b4 = f1.b;
        if (active) load_j(z_first, jx4, jy4, jz4);
    }
    Fill fn = load(zwrap(z_first + dz));

    for (int rel = 0; rel < L; rel++) {
        const int z = z_first + rel * dz;
        store(zwrap(z + dz), (rel + 2) & 3, fn);
        const float4 an = fn.a, bn = fn.b;               // own densities of plane z + 1
        if (rel + 1 < L) fn = load(zwrap(z + 2 * dz));
        if (active && rel > 0) load_j(z, jx4, jy4, jz4);
        __syncthreads();
        if (active)
            collide4_plane<MODE, T>(p, D, ring, plane_sz, rel, dz, r, x, ry, z, a4, b4, jx4, jy4, jz4, Fibm, mask,
                                    u_out, err);
        a4 = an;
        b4 = bn;
    }
}

// ------------------------------------------------------------------------------------------------------
// Staged forms: the inputs arrive in shared memory by bulk asynchronous copies (async_copy.cuh)
// ------------------------------------------------------------------------------------------------------
// Shared-memory loads of one storage element and of four consecutive ones (16-byte aligned for FP32, 8 for
// the 16-bit types).
__device__ __forceinline__ float sld(const float* p) { return *p; }
__device__ __forceinline__ float sld(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float sld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float4 sld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 sld4(const __half* p) {
    const __half2* h = reinterpret_cast<const __half2*>(p);
    const float2 a = __half22float2(h[0]), b = __half22float2(h[1]);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 sld4(const __nv_bfloat16* p) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(p);
    const float2 a = __bfloat1622float2(h[0]), b = __bfloat1622float2(h[1]);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float sld(const DevH* p) { return sld(raw16(p)); }
__device__ __forceinline__ float sld(const DevB* p) { return sld(raw16(p)); }
__device__ __forceinline__ float4 sld4(const DevH* p) { return sld4(raw16(p)); }
__device__ __forceinline__ float4 sld4(const DevB* p) { return sld4(raw16(p)); }

// the values direction I brings to the nodes x .. x+3 from a whole source row in shared memory (periodic in x)
template <int I, typename T>
__device__ __forceinline__ float4 srow4(const T* row, int x, int nx) {
    const float4 v = sld4(row + x);
    if (dir_x(I) == 1) return make_float4(sld(row + (x == 0 ? nx - 1 : x - 1)), v.x, v.y, v.z);
    if (dir_x(I) == -1) return make_float4(v.y, v.z, v.w, sld(row + (x + 4 == nx ? 0 : x + 4)));
    return v;
}

template <typename T, int I, int... Rest>
__device__ __forceinline__ void srow_all(const LbmParams& p, const T* stage, int x, int nx, Mom4& m,
                                         DirList<I, Rest...>) {
    float4 a = srow4<I, T>(stage + (size_t)I * nx, x, nx), b = srow4<I, T>(stage + (size_t)(Q + I) * nx, x, nx);
    if constexpr (is_dev<T>::value) {                  // deviation storage: add the reference back
        const float ra = dir_w(I) * p.rref[0], rb = dir_w(I) * p.rref[1];
        a = make_float4(a.x + ra, a.y + ra, a.z + ra, a.w + ra);
        b = make_float4(b.x + rb, b.y + rb, b.z + rb, b.w + rb);
    }
    acc_dir<I>(m, a, b);
    if constexpr (sizeof...(Rest) > 0) srow_all<T>(p, stage, x, nx, m, DirList<Rest...>{});
}

constexpr long long DRAIN_POLLS = 1LL << 22;     // bounded wait for the copies in flight after a give-up

// Kernel A, staged: every warp streams lattice rows (y, z), two in flight.  The 2 Q source rows of row (y, z)
// (direction i of component c pulls the whole row (y - c_y, z - c_z) of S[c][i]; the x-shift becomes an index
// into shared memory) arrive by cp.async.bulk on the warp's own mbarrier while the warp sums the previous row.
// The moments are the quad form's, summed in the same order, so both forms give the same bits.  A wait that
// gives up (p.wait_limit polls) raises bit 4 of the device error word; the warp lets its copies land and leaves.
template <typename T>
__global__ void __launch_bounds__(256) k_moments_staged(LbmParams p, const T* __restrict__ S, float* __restrict__ rho,
                                                        float* __restrict__ J, int* __restrict__ err) {
    pdl_wait();
    extern __shared__ __align__(128) unsigned char msm[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int nx = p.nx;
    const size_t stage_elems = (size_t)2 * Q * nx;
    uint64_t* bars = reinterpret_cast<uint64_t*>(msm) + 2 * w;
    T* stg = reinterpret_cast<T*>(msm + 128) + (size_t)w * 2 * stage_elems;
    const unsigned int rows = (unsigned)p.ny * (unsigned)(p.zf1 - p.zf0);
    const unsigned int stride = gridDim.x * (unsigned)wpb;
    unsigned int row = blockIdx.x * (unsigned)wpb + (unsigned)w;
    if (row >= rows) return;                             // the warp has no row (it never initialised a barrier)
    if (lane == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
    }
    __syncwarp();
    const uint32_t rowb = (uint32_t)(nx * sizeof(T));
    auto issue = [&](unsigned int rw, int b) {
        const int y = (int)(rw % (unsigned)p.ny), z = p.zf0 + (int)(rw / (unsigned)p.ny);
        T* sb = stg + (size_t)b * stage_elems;
        if (lane == 0) mbar_arrive_expect_tx(bars + b, 2u * Q * rowb);
        __syncwarp();
        if (lane < Q) {
            fence_proxy_async_smem();
            const int i = lane;
            int ys = y - dir_y(i), zs = z - dir_z(i);
            ys = ys < 0 ? ys + p.ny : (ys >= p.ny ? ys - p.ny : ys);
            if (!p.walls) zs = zs < 0 ? zs + p.nz : (zs >= p.nz ? zs - p.nz : zs);
            const size_t src = (size_t)ys * nx + (size_t)zs * p.nxy;
            bulk_g2s(sb + (size_t)i * nx, S + (size_t)i * p.N + src, rowb, bars + b);
            bulk_g2s(sb + (size_t)(Q + i) * nx, S + (size_t)(Q + i) * p.N + src, rowb, bars + b);
        }
    };
    uint32_t ph = 0u, pend = 1u;                        // bit b: the parity awaited on buffer b, copies pending
    int b = 0;
    issue(row, 0);
    for (; row < rows; row += stride) {
        const unsigned int nxt = row + stride;
        if (nxt < rows) {
            issue(nxt, b ^ 1);
            pend |= 2u >> b;
        }
        const bool ok = mbar_wait(bars + b, (ph >> b) & 1u, p.wait_limit);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                atomicOr(err, 4);
                for (int k = 0; k < 2; k++)
                    if ((pend >> k) & 1u) mbar_wait(bars + k, (ph >> k) & 1u, DRAIN_POLLS);
            }
            __syncwarp();
            return;
        }
        ph ^= 1u << b;
        pend &= ~(1u << b);
        const int y = (int)(row % (unsigned)p.ny), z = p.zf0 + (int)(row / (unsigned)p.ny);
        const T* sb = stg + (size_t)b * stage_elems;
        for (int q = lane; q < (nx >> 2); q += 32) {
            const int x = 4 * q;
            Mom4 m;
#pragma unroll
            for (int k = 0; k < 4; k++) m.ra[k] = m.rb[k] = m.jx[k] = m.jy[k] = m.jz[k] = 0.f;
            srow_all<T>(p, sb, x, nx, m, AllDirs{});
            const unsigned int n0 = (unsigned)x + (unsigned)y * nx + (unsigned)z * p.nxy;
            *reinterpret_cast<float4*>(rho + n0) = make_float4(m.ra[0], m.ra[1], m.ra[2], m.ra[3]);
            *reinterpret_cast<float4*>(rho + p.N + n0) = make_float4(m.rb[0], m.rb[1], m.rb[2], m.rb[3]);
            *reinterpret_cast<float4*>(J + n0) = make_float4(m.jx[0], m.jx[1], m.jx[2], m.jx[3]);
            *reinterpret_cast<float4*>(J + p.N + n0) = make_float4(m.jy[0], m.jy[1], m.jy[2], m.jy[3]);
            *reinterpret_cast<float4*>(J + 2 * (size_t)p.N + n0) = make_float4(m.jz[0], m.jz[1], m.jz[2], m.jz[3]);
        }
        __syncwarp();                                    // buffer b is read out before it is issued again
        b ^= 1;
    }
}

// Kernel B, staged: the collide4_tile march with its inputs delivered by bulk copies, which the first warp
// issues one plane ahead, so no thread waits on a global load inside the march.  Ring planes P_k = P_0 + k dz
// (P_0 = z_first - dz) arrive as stages k, in buffer k % 2: rho^A, rho^B of the tile rows and both halo rows
// of P_k (none for a wall plane, whose ghost densities are computed from the adjacent fluid plane as in the
// unstaged form) and, for k >= 2, j of the plane P_{k-1} that iteration k - 2 collides.  A buffer:
// [rho^A: TY + 2 rows][rho^B: TY + 2 rows][j_x: TY rows][j_y: TY rows][j_z: TY rows], rows of nx floats.
// The collision is collide4_plane on the same ring, so the results equal the unstaged form's bit for bit.  A
// wait that gives up raises bit 4 of the device error word; the block lets its copies land and leaves.
template <int MODE, typename T>
__device__ __forceinline__ void collide4_staged(const LbmParams& p, T* __restrict__ D, const float* __restrict__ rho,
                                                const float* __restrict__ J, float* __restrict__ ghost,
                                                const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
                                                float* __restrict__ u_out, int* __restrict__ err, int TY, int tile,
                                                int seg, int nseg, float* ring, float* stage, uint64_t* bar) {
    const int nx = p.nx;
    const int NQ = nx >> 2;
    const int RR = TY + 2;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int nreal = NQ * TY;
    const int tr = t < nreal ? t : nreal - 1;
    const int r = tr / NQ + 1;
    const int q = tr - (r - 1) * NQ;
    const int x = 4 * q;
    const int y0 = tile * TY;
    const int gy = y0 + r - 1;
    const bool active = t < nreal && gy < p.ny;
    const int plane_sz = RR * nx;
    const size_t stage_sz = (size_t)(2 * RR + 3 * TY) * nx;
    const int nJ = TY < p.ny - y0 ? TY : p.ny - y0;      // tile rows inside the lattice
    const int ry[3] = {(gy == 0 ? p.ny - 1 : gy - 1) * nx, gy * nx, (gy + 1 >= p.ny ? 0 : gy + 1) * nx};

    const int nzf = p.zf1 - p.zf0;
    const int zs = p.zf0 + (int)(((long long)seg * nzf) / nseg);
    const int ze = p.zf0 + (int)(((long long)(seg + 1) * nzf) / nseg);
    if (zs >= ze) return;
    const int dz = (seg & 1) ? 1 : -1;
    const int z_first = dz > 0 ? zs : ze - 1;
    const int L = ze - zs;
    auto zwrap = [&](int z) { return p.walls ? z : (z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z)); };
    auto plane_k = [&](int k) { return zwrap(z_first + (k - 1) * dz); };

    const bool own_q = t < nreal;
    const bool halo_q = t < 2 * NQ;
    const int hr = t < NQ ? 0 : TY + 1;
    const int hx = 4 * (t < NQ ? t : t - NQ);
    int hy = hr == 0 ? y0 - 1 : y0 + TY;
    hy = hy < 0 ? hy + p.ny : (hy >= p.ny ? hy - p.ny : hy);
    const int gyw = gy >= p.ny ? gy - p.ny : gy;

    if (t == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
    }
    __syncthreads();
    uint32_t ph = 0u, pend = 0u;                        // bit b: the parity awaited on buffer b, copies pending
    // the first warp issues stage k into buffer k % 2 (the buffer's previous contents were read before the
    // block barrier that precedes every call)
    auto issue = [&](int k) {
        const int b = k & 1;
        pend |= 1u << b;
        if (t >= 32) return;
        float* sb = stage + (size_t)b * stage_sz;
        const int zr = plane_k(k);
        const bool rows = !is_wall_plane(p, zr);
        const bool jrows = k >= 2;
        const uint32_t rowb = (uint32_t)nx * 4u;
        const uint32_t bytes = (rows ? 2u * RR * rowb : 0u) + (jrows ? 3u * (uint32_t)nJ * rowb : 0u);
        if (lane == 0) mbar_arrive_expect_tx(bar + b, bytes);
        __syncwarp();
        const int nc = (rows ? 2 * RR : 0) + (jrows ? 3 : 0);
        for (int c = lane; c < nc; c += 32) {
            fence_proxy_async_smem();
            if (rows && c < 2 * RR) {
                const int comp = c / RR, rr = c - comp * RR;
                int yy = y0 - 1 + rr;
                yy = yy < 0 ? yy + p.ny : (yy >= p.ny ? yy - p.ny : yy);
                bulk_g2s(sb + (size_t)(comp * RR + rr) * nx,
                         rho + (size_t)comp * p.N + (size_t)zr * p.nxy + (size_t)yy * nx, rowb, bar + b);
            } else {
                const int d = c - (rows ? 2 * RR : 0);
                bulk_g2s(sb + (size_t)(2 * RR + d * TY) * nx,
                         J + (size_t)d * p.N + (size_t)plane_k(k - 1) * p.nxy + (size_t)y0 * nx, (uint32_t)nJ * rowb,
                         bar + b);
            }
        }
    };
    auto wait = [&](int k) {
        const int b = k & 1;
        const bool ok = mbar_wait(bar + b, (ph >> b) & 1u, p.wait_limit);
        if (ok) {
            ph ^= 1u << b;
            pend &= ~(1u << b);
        }
        return ok;
    };
    auto give_up = [&]() {
        if (t == 0) {
            atomicOr(err, 4);
            for (int k = 0; k < 2; k++)
                if ((pend >> k) & 1u) mbar_wait(bar + k, (ph >> k) & 1u, DRAIN_POLLS);
        }
    };
    auto psi4 = [&](float4 v) {
        return make_float4(psi_fn(v.x, p.psi_kind), psi_fn(v.y, p.psi_kind), psi_fn(v.z, p.psi_kind),
                           psi_fn(v.w, p.psi_kind));
    };
    // ring slot `slot` <- psi of plane P_k from stage k (a wall plane: the ghost densities, computed and, by the
    // CTA that owns the rows, written out); the thread's own densities of P_k to oa, ob
    auto fill = [&](int k, int slot, float4& oa, float4& ob) {
        const float* sb = stage + (size_t)(k & 1) * stage_sz;
        const int zr = plane_k(k);
        float* base = ring + (size_t)slot * 2 * plane_sz;
        const bool wall = is_wall_plane(p, zr);
        const int za = zr == 0 ? 1 : p.nz - 2;
        if (own_q) {
            float4 a, bb;
            if (wall) {
                a = wall_ghost4(p, rho, x, gyw, za);
                bb = wall_ghost4(p, rho + p.N, x, gyw, za);
                if (active) {
                    const int w = zr == 0 ? 0 : 1;
                    *reinterpret_cast<float4*>(ghost + (w * 2 + 0) * p.nxy + gy * nx + x) = a;
                    *reinterpret_cast<float4*>(ghost + (w * 2 + 1) * p.nxy + gy * nx + x) = bb;
                }
            } else {
                a = *reinterpret_cast<const float4*>(sb + (size_t)r * nx + x);
                bb = *reinterpret_cast<const float4*>(sb + (size_t)(RR + r) * nx + x);
            }
            *reinterpret_cast<float4*>(base + r * nx + x) = psi4(a);
            *reinterpret_cast<float4*>(base + plane_sz + r * nx + x) = psi4(bb);
            oa = a;
            ob = bb;
        }
        if (halo_q) {
            float4 ha, hb;
            if (wall) {
                ha = wall_ghost4(p, rho, hx, hy, za);
                hb = wall_ghost4(p, rho + p.N, hx, hy, za);
            } else {
                ha = *reinterpret_cast<const float4*>(sb + (size_t)hr * nx + hx);
                hb = *reinterpret_cast<const float4*>(sb + (size_t)(RR + hr) * nx + hx);
            }
            *reinterpret_cast<float4*>(base + hr * nx + hx) = psi4(ha);
            *reinterpret_cast<float4*>(base + plane_sz + hr * nx + hx) = psi4(hb);
        }
    };

    float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f), b4 = a4, an = a4, bn = a4;
    issue(0);
    issue(1);
    bool ok = wait(0);
    fill(0, 0, an, bn);
    ok = wait(1) && ok;
    fill(1, 1, a4, b4);
    if (__syncthreads_or(!ok)) {
        give_up();
        return;
    }
    issue(2);                                            // buffer 0: stage 0 was read before the barrier
    for (int rel = 0; rel < L; rel++) {
        const int z = z_first + rel * dz;
        const int k = rel + 2;                           // stage of ring plane z + dz and of j of plane z
        ok = wait(k);
        fill(k, k & 3, an, bn);
        if (__syncthreads_or(!ok)) {
            give_up();
            return;
        }
        if (k + 1 <= L + 1) issue(k + 1);                // buffer of stage k - 1, read out before the barrier
        if (active) {
            const float* jr = stage + (size_t)(k & 1) * stage_sz + (size_t)(2 * RR + r - 1) * nx + x;
            const float4 jx4 = *reinterpret_cast<const float4*>(jr);
            const float4 jy4 = *reinterpret_cast<const float4*>(jr + (size_t)TY * nx);
            const float4 jz4 = *reinterpret_cast<const float4*>(jr + (size_t)2 * TY * nx);
            collide4_plane<MODE, T>(p, D, ring, plane_sz, rel, dz, r, x, ry, z, a4, b4, jx4, jy4, jz4, Fibm, mask,
                                    u_out, err);
        }
        a4 = an;
        b4 = bn;
    }
}

// ------------------------------------------------------------------------------------------------------
// Kernels of one context
// ------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_moments4(LbmParams p, const T* __restrict__ S, float* __restrict__ rho,
                                                  float* __restrict__ J) {
    pdl_wait();
    const unsigned int total = (unsigned)(p.nx >> 2) * (unsigned)p.ny * (unsigned)(p.zf1 - p.zf0);
    // a warp wholly past the end has nothing to do (it is never a shuffle partner of a live lane)
    if (blockIdx.x * blockDim.x + (threadIdx.x & ~31u) >= total) return;
    moments4_quad<T>(p, S, rho, J, blockIdx.x * blockDim.x + threadIdx.x, total);
}

template <typename T>
__global__ void __launch_bounds__(256) k_moments1(LbmParams p, const T* __restrict__ S, float* __restrict__ rho,
                                                  float* __restrict__ J) {
    pdl_wait();
    const unsigned int total = (unsigned)p.nx * (unsigned)p.ny * (unsigned)(p.zf1 - p.zf0);
    moments1_node<T>(p, S, rho, J, blockIdx.x * blockDim.x + threadIdx.x, total);
}

// one compiled kernel per form serves every block shape (at most 512 threads, 128 registers), so the
// per-node arithmetic, and the results, do not depend on the shape
template <int MODE, typename T, bool VEC>
__global__ void __launch_bounds__(512, 1)
k_collide(LbmParams p, T* __restrict__ D, const float* __restrict__ rho, const float* __restrict__ J,
          float* __restrict__ ghost, const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
          float* __restrict__ u_out, int* __restrict__ err, int TY) {
    pdl_wait();
    extern __shared__ float ring[];                      // psi [4 planes][2 components][TY + 2 rows][nx]
    if (VEC)
        collide4_tile<MODE, T>(p, D, rho, J, ghost, Fibm, mask, u_out, err, TY, blockIdx.x, blockIdx.y, gridDim.y,
                               ring);
    else
        collide1_tile<MODE, T>(p, D, rho, J, ghost, Fibm, mask, u_out, err, TY, blockIdx.x, blockIdx.y, gridDim.y,
                               ring);
}

// ---- Pair form of kernel B: two threads per quad, one per component (lanes 2j and 2j + 1 hold components A
// and B of the same four nodes).  A thread forms the force on its own component c only, which needs the
// gradient of the other component's psi (Eq. 13) and its own psi, and stores only its own component's f_eq,
// so it carries half the state of the quad form; every value it computes is the quad form's for that
// component, by the same operations in the same order, so the results are the same bits.
template <int MODE, typename T>
__device__ __forceinline__ void collide4_half(const LbmParams& p, T* __restrict__ D, const float* ring, int plane_sz,
                                              int rel, int dz, int r, int x, int c, const int ry[3], int z,
                                              float4 a4, float4 b4, float4 jx4, float4 jy4, float4 jz4,
                                              const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
                                              float* __restrict__ u_out, int* __restrict__ err, unsigned int pairs) {
    constexpr bool IBM = MODE == 1;
    const int nx = p.nx;
    const unsigned int n0 = (unsigned)x + (unsigned)ry[1] + (unsigned)z * p.nxy;
    const int s_back = rel & 3, s_ahead = (rel + 2) & 3;
    const float* pm = ring + (size_t)(dz > 0 ? s_back : s_ahead) * 2 * plane_sz;   // plane z - 1
    const float* p0 = ring + (size_t)((rel + 1) & 3) * 2 * plane_sz;               // plane z
    const float* pp = ring + (size_t)(dz > 0 ? s_ahead : s_back) * 2 * plane_sz;   // plane z + 1
    // gradient sums of the other component's psi (the quad form's S of component 1 - c)
    float So[3][4], ps[4];
    {
        const int co = (1 - c) * plane_sz;
        float w00[6], wyp[6], wym[6], wzp[6], wzm[6];
        window6(p0 + co + r * nx, x, nx, w00);
        window6(p0 + co + (r + 1) * nx, x, nx, wyp);
        window6(p0 + co + (r - 1) * nx, x, nx, wym);
        window6(pp + co + r * nx, x, nx, wzp);
        window6(pm + co + r * nx, x, nx, wzm);
        const float4 cpp = *reinterpret_cast<const float4*>(pp + co + (r + 1) * nx + x);
        const float4 cmp = *reinterpret_cast<const float4*>(pp + co + (r - 1) * nx + x);
        const float4 cpm = *reinterpret_cast<const float4*>(pm + co + (r + 1) * nx + x);
        const float4 cmm = *reinterpret_cast<const float4*>(pm + co + (r - 1) * nx + x);
        const float Cpp[4] = {cpp.x, cpp.y, cpp.z, cpp.w}, Cmp[4] = {cmp.x, cmp.y, cmp.z, cmp.w};
        const float Cpm[4] = {cpm.x, cpm.y, cpm.z, cpm.w}, Cmm[4] = {cmm.x, cmm.y, cmm.z, cmm.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            So[0][k] = (w00[k + 2] - w00[k]) * (1.f / 18.f) +
                       ((wyp[k + 2] - wyp[k]) + (wym[k + 2] - wym[k]) + (wzp[k + 2] - wzp[k]) +
                        (wzm[k + 2] - wzm[k])) * (1.f / 36.f);
            const float ty = (wyp[k + 2] + wyp[k]) - (wym[k + 2] + wym[k]);
            const float tz = (wzp[k + 2] + wzp[k]) - (wzm[k + 2] + wzm[k]);
            So[1][k] = (wyp[k + 1] - wym[k + 1]) * (1.f / 18.f) +
                       (ty + ((Cpp[k] + Cpm[k]) - (Cmp[k] + Cmm[k]))) * (1.f / 36.f);
            So[2][k] = (wzp[k + 1] - wzm[k + 1]) * (1.f / 18.f) +
                       (tz + ((Cpp[k] + Cmp[k]) - (Cpm[k] + Cmm[k]))) * (1.f / 36.f);
        }
        const float4 own = *reinterpret_cast<const float4*>(p0 + c * plane_sz + r * nx + x);
        ps[0] = own.x; ps[1] = own.y; ps[2] = own.z; ps[3] = own.w;
    }
    uint32_t bits = 0;
    if (IBM) bits = (__ldg(mask + (n0 >> 5)) >> (n0 & 31)) & 0xFu;
    const float ra[4] = {a4.x, a4.y, a4.z, a4.w}, rb[4] = {b4.x, b4.y, b4.z, b4.w};
    const float jxa[4] = {jx4.x, jx4.y, jx4.z, jx4.w}, jya[4] = {jy4.x, jy4.y, jy4.z, jy4.w},
                jza[4] = {jz4.x, jz4.y, jz4.z, jz4.w};
    float v[4][3], a[4], rc[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        rc[k] = c == 0 ? ra[k] : rb[k];
        const float rt = ra[k] + rb[k];
        const float irt = 1.f / rt;
        float F[3];
#pragma unroll
        for (int d = 0; d < 3; d++) F[d] = -ps[k] * p.G * So[d][k] + rc[k] * p.g[d];
        if (IBM && ((bits >> k) & 1u)) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const float fi = ibm_unfix(Fibm[(size_t)d * p.N + n0 + k]);
                F[d] += rc[k] * irt * fi;
            }
        }
        const float ux = jxa[k] * irt, uy = jya[k] * irt, uz = jza[k] * irt;
        if (!(rt > 0.f) || !(ux * ux + uy * uy + uz * uz <= 0.09f)) atomicOr(err, 1);
        const float tc = rc[k] > 0.f ? p.tau / rc[k] : 0.f;
        const float u0 = ux + tc * F[0], u1 = uy + tc * F[1], u2 = uz + tc * F[2];
        a[k] = 1.f - 1.5f * (u0 * u0 + u1 * u1 + u2 * u2);
        v[k][0] = 3.f * u0; v[k][1] = 3.f * u1; v[k][2] = 3.f * u2;
        if (IBM) {
            // the half-force velocity (j + (F^A + F^B) / 2) / rho at marked nodes: the A lane adds its
            // partner's force (the quad form's order, F^A + F^B); `pairs` holds both lanes of every pair here
            float Fo[3];
#pragma unroll
            for (int d = 0; d < 3; d++) Fo[d] = __shfl_xor_sync(pairs, F[d], 1);
            if (c == 0 && ((bits >> k) & 1u)) {
                u_out[n0 + k] = (jxa[k] + 0.5f * (F[0] + Fo[0])) * irt;
                u_out[(size_t)p.N + n0 + k] = (jya[k] + 0.5f * (F[1] + Fo[1])) * irt;
                u_out[(size_t)2 * p.N + n0 + k] = (jza[k] + 0.5f * (F[2] + Fo[2])) * irt;
            }
        }
    }
    // equilibrium (Eq. 2) of component c = its post-collision populations, by opposite-direction pairs
    const bool wall_next = p.walls && (z == 1 || z == p.nz - 2);
    T* Dc = D + (size_t)c * Q * p.N;
    float sc[4];
#pragma unroll
    for (int k = 0; k < 4; k++) sc[k] = 0.f;
    auto store_dir = [&](auto Ic, const float (&o)[4]) {
        constexpr int I = decltype(Ic)::value;
        if (dir_z(I) != 0 && wall_next && is_wall_plane(p, z + dir_z(I))) {
            // half-way bounce-back on a moving wall (Eq. 11), stored where the node pulls opp(I) from
            const float* U = (z + dir_z(I) == 0) ? p.ulo : p.uhi;
            const float cU = 6.f * dir_w(I) * (dir_x(I) * U[0] + dir_y(I) * U[1] + dir_z(I) * U[2]);
            const unsigned int drow = (unsigned)ry[1 + dir_y(I)] + (unsigned)(z + dir_z(I)) * p.nxy;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                int xd = x + k + dir_x(I);
                xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
                pst(Dc + (size_t)dir_opp(I) * p.N + drow + xd, o[k] - cU * rc[k]);
            }
        } else {
            pst4(Dc + (size_t)I * p.N + n0, make_float4(o[0], o[1], o[2], o[3]));
        }
    };
    auto emit_pair = [&](auto Ic) {
        constexpr int I = decltype(Ic)::value;
        constexpr float W = dir_w(I);
        float o[4], om[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float qv = cdot<I>(v[k][0], v[k][1], v[k][2]);
            const float h = fmaf(0.5f * qv, qv, a[k]);
            const float w = W * rc[k];
            if constexpr (is_dev<T>::value) {          // deviations from W rref^c
                const float dc = W * p.rref[c];
                o[k] = pround(w * (h + qv) - dc, D);
                om[k] = pround(w * (h - qv) - dc, D);
            } else {
                o[k] = pround(w * (h + qv), D);
                om[k] = pround(w * (h - qv), D);
            }
            sc[k] += o[k] + om[k];
        }
        store_dir(std::integral_constant<int, I>{}, o);
        store_dir(std::integral_constant<int, I + 1>{}, om);
    };
    emit_pair(std::integral_constant<int, 1>{});  emit_pair(std::integral_constant<int, 3>{});
    emit_pair(std::integral_constant<int, 5>{});  emit_pair(std::integral_constant<int, 7>{});
    emit_pair(std::integral_constant<int, 9>{});  emit_pair(std::integral_constant<int, 11>{});
    emit_pair(std::integral_constant<int, 13>{}); emit_pair(std::integral_constant<int, 15>{});
    emit_pair(std::integral_constant<int, 17>{});
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        o[k] = (rc[k] - dev_ref<T>(p, c)) - sc[k];
        if (sizeof(T) == 2) {
            const uint32_t h = dither_bits(n0 + k, ra[k], rb[k]);
            o[k] = pdither(o[k], c == 0 ? h >> 16 : h & 0xffffu, D);
        }
    }
    store_dir(std::integral_constant<int, 0>{}, o);
}

// The staged march of the pair form: thread t takes component t & 1 of quad t >> 1 of the tile (tile rows of
// nx / 4 quads); the stages, ring and waits are collide4_staged's, each thread filling its own component.
template <int MODE, typename T>
__device__ __forceinline__ void collide_pair_staged(const LbmParams& p, T* __restrict__ D, const float* __restrict__ rho,
                                                    const float* __restrict__ J, float* __restrict__ ghost,
                                                    const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
                                                    float* __restrict__ u_out, int* __restrict__ err, int TY, int tile,
                                                    int seg, int nseg, float* ring, float* stage, uint64_t* bar) {
    const int nx = p.nx;
    const int NQ = nx >> 2;
    const int RR = TY + 2;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int c = t & 1;
    const int t2 = t >> 1;
    const int nreal = NQ * TY;                           // quads of the tile
    const int tr = t2 < nreal ? t2 : nreal - 1;
    const int r = tr / NQ + 1;
    const int q = tr - (r - 1) * NQ;
    const int x = 4 * q;
    const int y0 = tile * TY;
    const int gy = y0 + r - 1;
    const bool own_q = t2 < nreal;
    const bool active = own_q && gy < p.ny;
    const int plane_sz = RR * nx;
    const size_t stage_sz = (size_t)(2 * RR + 3 * TY) * nx;
    const int nJ = TY < p.ny - y0 ? TY : p.ny - y0;
    const int ry[3] = {(gy == 0 ? p.ny - 1 : gy - 1) * nx, gy * nx, (gy + 1 >= p.ny ? 0 : gy + 1) * nx};

    const int nzf = p.zf1 - p.zf0;
    const int zs = p.zf0 + (int)(((long long)seg * nzf) / nseg);
    const int ze = p.zf0 + (int)(((long long)(seg + 1) * nzf) / nseg);
    if (zs >= ze) return;
    const int dz = (seg & 1) ? 1 : -1;
    const int z_first = dz > 0 ? zs : ze - 1;
    const int L = ze - zs;
    auto zwrap = [&](int z) { return p.walls ? z : (z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z)); };
    auto plane_k = [&](int k) { return zwrap(z_first + (k - 1) * dz); };

    const bool halo_q = t2 < 2 * NQ;
    const int hr = t2 < NQ ? 0 : TY + 1;
    const int hx = 4 * (t2 < NQ ? t2 : t2 - NQ);
    int hy = hr == 0 ? y0 - 1 : y0 + TY;
    hy = hy < 0 ? hy + p.ny : (hy >= p.ny ? hy - p.ny : hy);
    const int gyw = gy >= p.ny ? gy - p.ny : gy;
    const float* rho_c = rho + (size_t)c * p.N;

    if (t == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
    }
    __syncthreads();
    uint32_t ph = 0u, pend = 0u;
    auto issue = [&](int k) {
        const int b = k & 1;
        pend |= 1u << b;
        if (t >= 32) return;
        float* sb = stage + (size_t)b * stage_sz;
        const int zr = plane_k(k);
        const bool rows = !is_wall_plane(p, zr);
        const bool jrows = k >= 2;
        const uint32_t rowb = (uint32_t)nx * 4u;
        const uint32_t bytes = (rows ? 2u * RR * rowb : 0u) + (jrows ? 3u * (uint32_t)nJ * rowb : 0u);
        if (lane == 0) mbar_arrive_expect_tx(bar + b, bytes);
        __syncwarp();
        const int nc = (rows ? 2 * RR : 0) + (jrows ? 3 : 0);
        for (int cc = lane; cc < nc; cc += 32) {
            fence_proxy_async_smem();
            if (rows && cc < 2 * RR) {
                const int comp = cc / RR, rr = cc - comp * RR;
                int yy = y0 - 1 + rr;
                yy = yy < 0 ? yy + p.ny : (yy >= p.ny ? yy - p.ny : yy);
                bulk_g2s(sb + (size_t)(comp * RR + rr) * nx,
                         rho + (size_t)comp * p.N + (size_t)zr * p.nxy + (size_t)yy * nx, rowb, bar + b);
            } else {
                const int d = cc - (rows ? 2 * RR : 0);
                bulk_g2s(sb + (size_t)(2 * RR + d * TY) * nx,
                         J + (size_t)d * p.N + (size_t)plane_k(k - 1) * p.nxy + (size_t)y0 * nx, (uint32_t)nJ * rowb,
                         bar + b);
            }
        }
    };
    auto wait = [&](int k) {
        const int b = k & 1;
        const bool ok = mbar_wait(bar + b, (ph >> b) & 1u, p.wait_limit);
        if (ok) {
            ph ^= 1u << b;
            pend &= ~(1u << b);
        }
        return ok;
    };
    auto give_up = [&]() {
        if (t == 0) {
            atomicOr(err, 4);
            for (int k = 0; k < 2; k++)
                if ((pend >> k) & 1u) mbar_wait(bar + k, (ph >> k) & 1u, DRAIN_POLLS);
        }
    };
    auto psi4 = [&](float4 v) {
        return make_float4(psi_fn(v.x, p.psi_kind), psi_fn(v.y, p.psi_kind), psi_fn(v.z, p.psi_kind),
                           psi_fn(v.w, p.psi_kind));
    };
    // ring slot `slot` <- psi of component c of plane P_k; both components' own densities to oa, ob
    auto fill = [&](int k, int slot, float4& oa, float4& ob) {
        const float* sb = stage + (size_t)(k & 1) * stage_sz;
        const int zr = plane_k(k);
        float* base = ring + (size_t)slot * 2 * plane_sz + (size_t)c * plane_sz;
        const bool wall = is_wall_plane(p, zr);
        const int za = zr == 0 ? 1 : p.nz - 2;
        if (own_q) {
            float4 a, bb;
            if (wall) {
                a = wall_ghost4(p, rho, x, gyw, za);
                bb = wall_ghost4(p, rho + p.N, x, gyw, za);
                if (active) {
                    const int w = zr == 0 ? 0 : 1;
                    *reinterpret_cast<float4*>(ghost + (w * 2 + c) * p.nxy + gy * nx + x) = c == 0 ? a : bb;
                }
            } else {
                a = *reinterpret_cast<const float4*>(sb + (size_t)r * nx + x);
                bb = *reinterpret_cast<const float4*>(sb + (size_t)(RR + r) * nx + x);
            }
            *reinterpret_cast<float4*>(base + r * nx + x) = psi4(c == 0 ? a : bb);
            oa = a;
            ob = bb;
        }
        if (halo_q) {
            float4 h;
            if (wall) h = wall_ghost4(p, rho_c, hx, hy, za);
            else h = *reinterpret_cast<const float4*>(sb + (size_t)(c * RR + hr) * nx + hx);
            *reinterpret_cast<float4*>(base + hr * nx + hx) = psi4(h);
        }
    };

    float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f), b4 = a4, an = a4, bn = a4;
    issue(0);
    issue(1);
    bool ok = wait(0);
    fill(0, 0, an, bn);
    ok = wait(1) && ok;
    fill(1, 1, a4, b4);
    if (__syncthreads_or(!ok)) {
        give_up();
        return;
    }
    issue(2);
    for (int rel = 0; rel < L; rel++) {
        const int z = z_first + rel * dz;
        const int k = rel + 2;
        ok = wait(k);
        fill(k, k & 3, an, bn);
        if (__syncthreads_or(!ok)) {
            give_up();
            return;
        }
        if (k + 1 <= L + 1) issue(k + 1);
        // both lanes of a pair are active or neither; the active pairs of the warp exchange forces by shuffle
        const unsigned int pairs = __ballot_sync(0xffffffffu, active);
        if (active) {
            const float* jr = stage + (size_t)(k & 1) * stage_sz + (size_t)(2 * RR + r - 1) * nx + x;
            const float4 jx4 = *reinterpret_cast<const float4*>(jr);
            const float4 jy4 = *reinterpret_cast<const float4*>(jr + (size_t)TY * nx);
            const float4 jz4 = *reinterpret_cast<const float4*>(jr + (size_t)2 * TY * nx);
            collide4_half<MODE, T>(p, D, ring, plane_sz, rel, dz, r, x, c, ry, z, a4, b4, jx4, jy4, jz4, Fibm,
                                   mask, u_out, err, pairs);
        }
        a4 = an;
        b4 = bn;
    }
}

template <int MODE, typename T>
__global__ void __launch_bounds__(256, 3)
k_collide_pair(LbmParams p, T* __restrict__ D, const float* __restrict__ rho, const float* __restrict__ J,
               float* __restrict__ ghost, const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
               float* __restrict__ u_out, int* __restrict__ err, int TY) {
    pdl_wait();
    extern __shared__ __align__(128) unsigned char psm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(psm);
    float* ring = reinterpret_cast<float*>(psm + 128);
    float* stage = ring + (size_t)4 * 2 * (TY + 2) * p.nx;
    collide_pair_staged<MODE, T>(p, D, rho, J, ghost, Fibm, mask, u_out, err, TY, blockIdx.x, blockIdx.y, gridDim.y,
                                 ring, stage, bar);
}

template <int MODE, typename T>
__global__ void __launch_bounds__(512, 1)
k_collide_staged(LbmParams p, T* __restrict__ D, const float* __restrict__ rho, const float* __restrict__ J,
                 float* __restrict__ ghost, const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
                 float* __restrict__ u_out, int* __restrict__ err, int TY) {
    pdl_wait();
    // [2 barriers, padded to 128 bytes][psi ring: 4 planes x 2 components x (TY + 2) rows x nx][2 stage buffers]
    extern __shared__ __align__(128) unsigned char csm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(csm);
    float* ring = reinterpret_cast<float*>(csm + 128);
    float* stage = ring + (size_t)4 * 2 * (TY + 2) * p.nx;
    collide4_staged<MODE, T>(p, D, rho, J, ghost, Fibm, mask, u_out, err, TY, blockIdx.x, blockIdx.y, gridDim.y,
                             ring, stage, bar);
}

// ------------------------------------------------------------------------------------------------------
// Geometry
// ------------------------------------------------------------------------------------------------------
// Shapes of kernel B: (threads per CTA, CTAs per SM, fewest planes per z-segment), chosen by b4cfg.
struct SplitShape {
    int nt, cps, min_planes;
};
static SplitShape split_shape(int cfg) {
    switch (cfg) {
        case 1: return {512, 1, 4};
        case 2: return {256, 2, 8};
        case 3: return {128, 4, 4};
        default: return {256, 2, 4};
    }
}

// Tile rows and threads of kernel B for a CTA of about nt threads: the quad form needs NQ = nx / 4 threads per
// row, the scalar form nx, and at least two rows' worth (the halo rows are filled by the first threads).
static bool split_rows(const LbmParams& p, int nt, int& TY, int& threads, bool& vec) {
    vec = p.nx % 4 == 0;
    const int per_row = vec ? p.nx / 4 : p.nx;
    if (2 * per_row > 512) return false;
    TY = std::max(1, std::min(nt / per_row, p.ny));
    threads = (std::max(per_row * TY, 2 * per_row) + 31) / 32 * 32;
    return threads <= 512;
}

bool bulk_split(const LbmParams& p) {
    if (bulk_variant() != 5 || p.omega != 1.0f) return false;
    int TY, th;
    bool vec;
    return split_rows(p, split_shape(p.b4cfg).nt, TY, th, vec);
}

static int split_segments(const LbmParams& p, int cols, int slots, int min_planes) {
    const int nzf = p.zf1 - p.zf0;
    int nseg = 1;
    double best = -1.0;
    for (int w = 1; w <= 4; w++) {
        int ns = (slots * w) / cols;
        if (ns < 1) ns = 1;
        const int cap = nzf / min_planes > 0 ? nzf / min_planes : 1;
        if (ns > cap) ns = cap;
        const int nb = cols * ns;
        const int waves = (nb + slots - 1) / slots;
        const double eff = (double)nb / ((double)slots * waves) - 0.02 * waves;
        if (eff > best + 1e-9) { best = eff; nseg = ns; }
    }
    return nseg;
}

static bool split_geometry(const LbmParams& p, dim3& grid, int& threads, int& TY, size_t& smem, bool& vec) {
    const SplitShape sh = split_shape(p.b4cfg);
    if (!split_rows(p, sh.nt, TY, threads, vec)) return false;
    const int cols = (p.ny + TY - 1) / TY;
    grid = dim3(cols, split_segments(p, cols, 152 * sh.cps, sh.min_planes), 1);
    smem = (size_t)4 * 2 * (TY + 2) * p.nx * sizeof(float);
    return true;
}

int split_grid_blocks(const LbmParams& p) {
    dim3 g;
    int th, ty;
    size_t sm;
    bool vec;
    return split_geometry(p, g, th, ty, sm, vec) ? (int)(g.x * g.y) : 0;
}

template <int MODE, typename T, bool VEC>
static void launch_collide(const LbmParams& p, dim3 grid, int threads, size_t smem, int TY, T* D, const float* rho,
                           const float* J, float* ghost, const IbmF* Fibm, const uint32_t* mask, float* u, int* err,
                           cudaStream_t st) {
    static size_t attr = 0;
    if (smem > attr) {
        cudaFuncSetAttribute(k_collide<MODE, T, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    launch_k(k_collide<MODE, T, VEC>, dim3(grid), dim3(threads), smem, st, p, D, rho, J, ghost, Fibm, mask, u, err, TY);
}

// The staged forms (bulk asynchronous copies into shared memory) serve quad rows; SCBB_BULK_STAGED=0 turns
// them off (the unstaged forms give the same bits).
static bool staged_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("SCBB_BULK_STAGED");
        v = (e && e[0] == '0' && e[1] == 0) ? 0 : 1;
    }
    return v == 1;
}

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    }
    return n;
}

constexpr size_t STAGED_SMEM_MAX = 227 * 1024;
constexpr size_t MOMENTS_SMEM_BUDGET = 200 * 1024;

// Kernel A staged: whole source rows of 16-byte multiples, rows long enough to be worth a copy each, no
// on-site velocity planes (their nodes reconstruct populations one by one).  Warps per CTA from the shared-
// memory budget (two row stages of 2 Q rows per warp).
static bool moments_staged_geometry(const LbmParams& p, int& wpb, size_t& smem) {
    const size_t es = p.store == 0 ? 4 : 2;
    if (!staged_enabled() || p.onsite || p.nx < 64 || p.nx > 512 || (p.nx * es) % 16 != 0) return false;
    const size_t two = 2 * (size_t)2 * Q * p.nx * es;
    wpb = (int)std::min<size_t>(8, (MOMENTS_SMEM_BUDGET - 128) / two);
    // fewer than four streaming warps per SM cannot keep the loads in flight (256-wide FP32 rows: two warps,
    // slower than the register form)
    if (wpb < 4) return false;
    smem = 128 + (size_t)wpb * two;
    return true;
}

static size_t collide_staged_smem(const LbmParams& p, int TY) {
    return 128 + (size_t)4 * 2 * (TY + 2) * p.nx * sizeof(float) + (size_t)2 * (2 * (TY + 2) + 3 * TY) * p.nx * sizeof(float);
}

// Kernel B, pair form: 256 threads, two per quad, TY tile rows (at least 2, so that the two halo rows'
// 4 nx / 4 fills have threads), three CTAs per SM.
constexpr int PAIR_THREADS = 256;
static bool pair_geometry(const LbmParams& p, dim3& grid, int& TY, size_t& smem) {
    if (!staged_enabled() || p.nx % 4 != 0) return false;
    const int NQ = p.nx / 4;
    if (4 * NQ > PAIR_THREADS) return false;
    TY = std::max(2, std::min(PAIR_THREADS / (2 * NQ), p.ny));
    if (2 * NQ * TY > PAIR_THREADS) return false;
    // tiles under four rows re-read their two halo rows for every one or two rows collided (nx > 128)
    if (TY < 4 && TY < p.ny) return false;
    const int cols = (p.ny + TY - 1) / TY;
    grid = dim3(cols, split_segments(p, cols, sm_count() * 3, 4), 1);
    smem = collide_staged_smem(p, TY);
    return smem <= STAGED_SMEM_MAX / 3;
}

static bool pair_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("SCBB_BULK_PAIR");
        v = (e && e[0] == '0' && e[1] == 0) ? 0 : 1;
    }
    return v == 1;
}

template <int MODE, typename T>
static void launch_collide_pair(const LbmParams& p, dim3 grid, size_t smem, int TY, T* D, const float* rho,
                                const float* J, float* ghost, const IbmF* Fibm, const uint32_t* mask, float* u,
                                int* err, cudaStream_t st) {
    static size_t attr = 0;
    if (smem > attr) {
        cudaFuncSetAttribute(k_collide_pair<MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    launch_k(k_collide_pair<MODE, T>, dim3(grid), dim3(PAIR_THREADS), smem, st, p, D, rho, J, ghost, Fibm, mask, u, err, TY);
}

template <typename T>
static void launch_moments_staged(const LbmParams& p, int wpb, size_t smem, const T* S, float* rho, float* J, int* err,
                                  cudaStream_t st) {
    static size_t attr = 0;
    static int per_sm = 0;
    if (smem > attr) {
        cudaFuncSetAttribute(k_moments_staged<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
        per_sm = 0;
    }
    if (per_sm == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_moments_staged<T>, 32 * wpb, smem) !=
                            cudaSuccess || per_sm < 1))
        per_sm = 1;
    const unsigned int rows = (unsigned)p.ny * (unsigned)(p.zf1 - p.zf0);
    const unsigned int need = (rows + wpb - 1) / wpb;
    const unsigned int blocks = std::min<unsigned int>(need, (unsigned)(sm_count() * per_sm));
    launch_k(k_moments_staged<T>, dim3(blocks), dim3(32 * wpb), smem, st, p, S, rho, J, err);
}

template <int MODE, typename T>
static void launch_collide_staged(const LbmParams& p, dim3 grid, int threads, size_t smem, int TY, T* D,
                                  const float* rho, const float* J, float* ghost, const IbmF* Fibm,
                                  const uint32_t* mask, float* u, int* err, cudaStream_t st) {
    static size_t attr = 0;
    if (smem > attr) {
        cudaFuncSetAttribute(k_collide_staged<MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    launch_k(k_collide_staged<MODE, T>, dim3(grid), dim3(threads), smem, st, p, D, rho, J, ghost, Fibm, mask, u, err, TY);
}

void launch_split(const LbmParams& p, const float* S, float* D, float* rho, float* J, float* ghost,
                  const IbmF* Fibm, const uint32_t* mask, float* u, int* err, int mode, cudaStream_t st) {
    dim3 grid;
    int threads, TY;
    size_t smem;
    bool vec;
    if (!split_geometry(p, grid, threads, TY, smem, vec)) return;
    const unsigned int units = (unsigned)(vec ? p.nx / 4 : p.nx) * p.ny * (p.zf1 - p.zf0);
    int wpb = 0;
    size_t msmem = 0;
    const bool a_staged = vec && moments_staged_geometry(p, wpb, msmem);
    const size_t csmem = collide_staged_smem(p, TY);
    // the staged quad form, like the pair form, where tiles hold at least four rows of at most 128 nodes
    const bool b_staged = vec && staged_enabled() && csmem <= STAGED_SMEM_MAX && p.nx <= 128;
    dim3 pgrid;
    int pTY = 0;
    size_t psmem = 0;
    const bool b_pair = vec && pair_enabled() && pair_geometry(p, pgrid, pTY, psmem);
    with_storage(p.store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        T* Dt = reinterpret_cast<T*>(D);
        if (vec) {
            if (a_staged) launch_moments_staged<T>(p, wpb, msmem, reinterpret_cast<const T*>(S), rho, J, err, st);
            else launch_k(k_moments4<T>, dim3((units + 255) / 256), dim3(256), 0, st, p, reinterpret_cast<const T*>(S), rho, J);
            if (b_pair) {
                if (mode == 1) launch_collide_pair<1, T>(p, pgrid, psmem, pTY, Dt, rho, J, ghost, Fibm, mask, u, err, st);
                else launch_collide_pair<0, T>(p, pgrid, psmem, pTY, Dt, rho, J, ghost, Fibm, mask, u, err, st);
            } else if (b_staged) {
                if (mode == 1) launch_collide_staged<1, T>(p, grid, threads, csmem, TY, Dt, rho, J, ghost, Fibm, mask, u, err, st);
                else launch_collide_staged<0, T>(p, grid, threads, csmem, TY, Dt, rho, J, ghost, Fibm, mask, u, err, st);
            } else if (mode == 1) {
                launch_collide<1, T, true>(p, grid, threads, smem, TY, Dt, rho, J, ghost, Fibm, mask, u, err, st);
            } else {
                launch_collide<0, T, true>(p, grid, threads, smem, TY, Dt, rho, J, ghost, Fibm, mask, u, err, st);
            }
        } else {
            launch_k(k_moments1<T>, dim3((units + 255) / 256), dim3(256), 0, st, p, reinterpret_cast<const T*>(S), rho, J);
            if (mode == 1) launch_collide<1, T, false>(p, grid, threads, smem, TY, Dt, rho, J, ghost, Fibm, mask, u, err, st);
            else launch_collide<0, T, false>(p, grid, threads, smem, TY, Dt, rho, J, ghost, Fibm, mask, u, err, st);
        }
    });
}

// ------------------------------------------------------------------------------------------------------
// Batches: one persistent cooperative launch for the bulk phase of every box
// ------------------------------------------------------------------------------------------------------
// Grid barrier with a bounded wait.  bar[0] counts the CTAs that arrived, bar[1] is the generation: the last CTA
// to arrive resets the count and advances the generation, the others wait for the generation to move.  Every CTA
// arrives exactly once, so the count is back at 0 after every use, timed out or not.  A wait that sees no
// progress within spin_limit polls (about 0.26 us each; none with a limit of 0) gives up: the CTA raises bit 4
// of every box's error word and the call returns false for the whole CTA.
__device__ bool grid_barrier(int* bar, long long spin_limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* gen = bar + 1;
        const int g = *gen;
        __threadfence();
        ok = 1;
        if (atomicAdd(bar, 1) == (int)gridDim.x - 1) {
            atomicExch(bar, 0);
            __threadfence();
            atomicAdd(bar + 1, 1);
        } else {
            // spin_limit polls at most, each after a short sleep; with a limit of 0 the wait gives up at once
            long long spins = 0;
            do {
                if (spins++ >= spin_limit) {
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            } while (*gen == g);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256, 2) k_batch_bulk(const __grid_constant__ BatchDesc d) {
    extern __shared__ float ring[];
    // ---- kernel A of every box; each box's threads start at a multiple of 32, so no warp spans two boxes
    const unsigned int stride = gridDim.x * blockDim.x;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x;; g += stride) {
        const unsigned int wbase = g & ~31u;
        if (wbase >= d.a_total) break;
        int k = 0;
        while (k + 1 < d.nbox && d.box[k + 1].a_begin <= wbase) k++;
        const BatchBox& b = d.box[k];
        if (b.vec)
            moments4_quad<T>(b.p, static_cast<const T*>(b.S), b.rho, b.J, g - b.a_begin, b.a_count);
        else
            moments1_node<T>(b.p, static_cast<const T*>(b.S), b.rho, b.J, g - b.a_begin, b.a_count);
    }
    if (!grid_barrier(d.bar, d.spin_limit)) {
        if (threadIdx.x == 0)
            for (int k = 0; k < d.nbox; k++) atomicOr(d.box[k].err, 4);
        return;
    }
    // ---- kernel B of every box, one (tile, z-segment) item per CTA at a time
    for (int it = blockIdx.x; it < d.b_total; it += gridDim.x) {
        int k = 0;
        while (k + 1 < d.nbox && d.box[k + 1].b_begin <= it) k++;
        const BatchBox& b = d.box[k];
        const int loc = it - b.b_begin;
        const int tile = loc % b.cols, seg = loc / b.cols;
        if (b.vec)
            collide4_tile<MODE, T>(b.p, static_cast<T*>(b.D), b.rho, b.J, b.ghost, b.Fibm, b.mask, b.u, b.err, b.TY,
                                   tile, seg, b.nseg, ring);
        else
            collide1_tile<MODE, T>(b.p, static_cast<T*>(b.D), b.rho, b.J, b.ghost, b.Fibm, b.mask, b.u, b.err, b.TY,
                                   tile, seg, b.nseg, ring);
        __syncthreads();                    // the next item refills the ring
    }
}

// Fills the work layout of d (boxes already set: p, pointers) for CTAs of 256 threads; false if a box does not fit.
static bool batch_layout(BatchDesc& d, size_t& smem) {
    unsigned int a = 0;
    int items = 0;
    smem = 0;
    for (int k = 0; k < d.nbox; k++) {
        BatchBox& b = d.box[k];
        int threads;
        bool vec;
        if (!split_rows(b.p, BATCH_THREADS, b.TY, threads, vec) || threads > BATCH_THREADS) return false;
        b.vec = vec ? 1 : 0;
        b.a_begin = a;
        b.a_count = (unsigned)(vec ? b.p.nx / 4 : b.p.nx) * b.p.ny * (b.p.zf1 - b.p.zf0);
        a += (b.a_count + 31) / 32 * 32;
        b.cols = (b.p.ny + b.TY - 1) / b.TY;
        b.nseg = std::max(1, std::min(b.p.zf1 - b.p.zf0, (b.p.zf1 - b.p.zf0 + 7) / 8));
        b.b_begin = items;
        items += b.cols * b.nseg;
        smem = std::max(smem, (size_t)4 * 2 * (b.TY + 2) * b.p.nx * sizeof(float));
    }
    d.a_total = a;
    d.b_total = items;
    return true;
}

// Launches the bulk phase of all boxes of d as one cooperative kernel on st.  Returns false (nothing launched)
// when the boxes cannot share one launch.
bool launch_batch_bulk(BatchDesc& d, int mode, int store, cudaStream_t st) {
    size_t smem;
    if (d.nbox < 1 || d.nbox > BATCH_MAX || !batch_layout(d, smem)) return false;
    bool ok = false;
    with_storage(store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        const void* fn = mode == 1 ? (const void*)k_batch_bulk<T, 1> : (const void*)k_batch_bulk<T, 0>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BATCH_THREADS, smem) != cudaSuccess ||
            per_sm < 1)
            return;
        void* args[] = {&d};
        ok = cudaLaunchCooperativeKernel(fn, dim3(sms * per_sm), dim3(BATCH_THREADS), args, smem, st) == cudaSuccess;
    });
    if (!ok) cudaGetLastError();
    return ok;
}

}  // namespace scbb
