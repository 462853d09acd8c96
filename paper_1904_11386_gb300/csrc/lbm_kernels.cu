// Fluid kernels of libscbb: fused two-component stream + Shan-Chen force + BGK collide (Eq. 1-5, Eq. 13),
// half-way bounce-back walls (Eq. 11), initial state, exports and FP64 reductions.  sm_103a.
//
// Bulk kernel design.  The Shan-Chen force at x needs psi(rho) of all 18 neighbours at the same time level,
// and rho is only known after streaming.  Instead of a separate density pass (which would re-read all
// populations, +150 B per node), each CTA owns a TX x TY column of nodes and marches through a z-segment.
// For every plane it pulls the populations of its tile plus a one-node halo ring, sums them into rho^A,
// rho^B, and keeps psi of the last four planes in a shared-memory ring; the tile's own populations stay in
// registers for one plane and are collided once the plane above is known.  Halo pulls hit L2 (the
// neighbouring tile loaded them), so DRAM traffic stays at one read and one write of the populations plus
// the density write-out.
#include <math.h>
#include <stdlib.h>

#include <type_traits>

#include <algorithm>

#include "pull.cuh"
#include "scbb_internal.cuh"

namespace scbb {

// ------------------------------------------------------------------------------------------------------
// Initial state: every fluid node x writes f_eq,i(rho^c(x), u(x)) into the slot it pulls direction i from,
// (c, i, x - c_i); the rest population closes the node's mass over the values as stored.  The lattice is
// zeroed beforehand (slots only wall nodes would pull from stay 0).
// ------------------------------------------------------------------------------------------------------
template <typename T, typename TI>
__global__ void k_init_state(LbmParams p, T* __restrict__ S, const TI* __restrict__ rho_st,
                             const TI* __restrict__ u_st) {
    const unsigned int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const int z = n / p.nxy;
    if (is_wall_plane(p, z)) return;
    const int r = n - z * p.nxy;
    const int y = r / p.nx, x = r - y * p.nx;
    // the fields in FP32 (rounded to nearest when they come in FP64)
    const float ux = (float)u_st[n], uy = (float)u_st[p.N + n], uz = (float)u_st[2 * p.N + n];
    const float a = (float)rho_st[n], b = (float)rho_st[p.N + n];
    const float uu = ux * ux + uy * uy + uz * uz;
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const float cu = dir_x(i) * ux + dir_y(i) * uy + dir_z(i) * uz;
        const float e = dir_w(i) * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * uu);
        // a deviation storage keeps e rho - w_i rref^c (e carries w_i)
        const float va = pround(e * a - dir_w(i) * dev_ref<T>(p, 0), S), vb = pround(e * b - dir_w(i) * dev_ref<T>(p, 1), S);
        sa += va;
        sb += vb;
        int zs = z - dir_z(i);
        if (!p.walls) zs = wrapi(zs, p.nz);
        const unsigned int m = wrapi(x - dir_x(i), p.nx) + p.nx * (wrapi(y - dir_y(i), p.ny) + p.ny * zs);
        pst(S + (size_t)i * p.N + m, va);
        pst(S + (size_t)(Q + i) * p.N + m, vb);
    }
    const uint32_t h = dither_bits(n, a, b);
    pst(S + n, pdither((a - dev_ref<T>(p, 0)) - sa, h >> 16, S));
    pst(S + (size_t)Q * p.N + n, pdither((b - dev_ref<T>(p, 1)) - sb, h & 0xffffu, S));
}

// ------------------------------------------------------------------------------------------------------
// Virtual densities of the wall planes (neutral wetting): the wall node (x, y, 0) is seen with the mean
// density of its five fluid neighbours (x, y, 1), (x +- 1, y, 1), (x, y +- 1, 1); likewise at the top.
// ------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_wall_planes_rho(LbmParams p, const T* __restrict__ S, float* __restrict__ wall_rho) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2 * p.nxy) return;
    int w = q / p.nxy;
    int r = q - w * p.nxy;
    int y = r / p.nx, x = r - y * p.nx;
    int z = w == 0 ? 1 : p.nz - 2;
    Cols k;
    k.cx[0] = wrapi(x - 1, p.nx); k.cx[1] = x; k.cx[2] = wrapi(x + 1, p.nx);
    k.ry[0] = wrapi(y - 1, p.ny) * p.nx; k.ry[1] = y * p.nx; k.ry[2] = wrapi(y + 1, p.ny) * p.nx;
    float f[2 * Q];
    pull(p, S, k, z, f);
    float ra = 0.f, rb = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) { ra += f[i]; rb += f[Q + i]; }
    wall_rho[(w * 2 + 0) * p.nxy + r] = ra;
    wall_rho[(w * 2 + 1) * p.nxy + r] = rb;
}

__global__ void k_wall_ghost(LbmParams p, const float* __restrict__ wall_rho, float* __restrict__ ghost) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 4 * p.nxy) return;
    int wc = q / p.nxy;
    int r = q - wc * p.nxy;
    int y = r / p.nx, x = r - y * p.nx;
    const float* a = wall_rho + wc * p.nxy;
    float s = a[r] + a[wrapi(x - 1, p.nx) + y * p.nx] + a[wrapi(x + 1, p.nx) + y * p.nx] +
              a[x + wrapi(y - 1, p.ny) * p.nx] + a[x + wrapi(y + 1, p.ny) * p.nx];
    ghost[q] = s * 0.2f;
}

// Tile of the general bulk kernel: block = (TX+2)(TY+2) threads, TX*TY tile nodes first, then the halo ring.
template <int TX, int TY>
struct Tile {
    static constexpr int HX = TX + 2, HY = TY + 2, HN = HX * HY, NI = TX * TY;
};

// ------------------------------------------------------------------------------------------------------
// General bulk kernel (any nx; the path for tau != 1 when nx is not a multiple of 4).  Fused two-component
// pull, Shan-Chen force and collision on a TX x TY tile with a one-node halo ring, marching through a
// z-segment: each tile thread parks the populations it pulled for the next plane in shared memory (two
// planes, ping-pong, private to the thread) and streams the collision direction by direction, so two CTAs
// fit on an SM and one CTA's loads overlap the other's collision.
// ------------------------------------------------------------------------------------------------------
template <int TX, int TY>
constexpr int bulk2_smem_bytes() {
    return (4 * 2 * Tile<TX, TY>::HN + 2 * 2 * Q * Tile<TX, TY>::NI) * (int)sizeof(float);
}

template <int TX, int TY, bool IBM>
__global__ void __launch_bounds__(Tile<TX, TY>::HN, 2)
k_bulk2(LbmParams p, const float* __restrict__ S, float* __restrict__ D, float* __restrict__ rho_out,
        const float* __restrict__ ghost, const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
        float* __restrict__ u_out, int* __restrict__ err) {
    using T = Tile<TX, TY>;
    extern __shared__ float smem[];
    float* ring = smem;                                  // [4 planes][2 comp][HN]  psi
    float* hold = smem + 4 * 2 * T::HN;                  // [2 planes][2Q][NI]      pulled populations

    const int t = threadIdx.x;
    int lx, ly;
    if (t < T::NI) {
        lx = t % TX; ly = t / TX;
    } else {
        int h = t - T::NI;
        if (h < T::HX) { lx = h - 1; ly = -1; }
        else if (h < 2 * T::HX) { lx = h - T::HX - 1; ly = TY; }
        else if (h < 2 * T::HX + TY) { lx = -1; ly = h - 2 * T::HX; }
        else { lx = TX; ly = h - 2 * T::HX - TY; }
    }
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int gx = wrapi(x0 + lx, p.nx), gy = wrapi(y0 + ly, p.ny);
    const bool tile = t < T::NI;
    const bool active = tile && (x0 + lx < p.nx) && (y0 + ly < p.ny);
    const int si = (ly + 1) * T::HX + (lx + 1);

    Cols k;
    k.cx[0] = wrapi(gx - 1, p.nx); k.cx[1] = gx; k.cx[2] = wrapi(gx + 1, p.nx);
    k.ry[0] = wrapi(gy - 1, p.ny) * p.nx; k.ry[1] = gy * p.nx; k.ry[2] = wrapi(gy + 1, p.ny) * p.nx;

    const int zs = p.zf0 + blockIdx.z * p.lz;
    const int ze = min(zs + p.lz, p.zf1);
    if (zs >= ze) return;

    auto plane = [&](int z, int slot, int buf) {
        if (is_wall_plane(p, z)) {
            const int w = z == 0 ? 0 : 1;
            const int r = gx + gy * p.nx;
            ring[(slot * 2 + 0) * T::HN + si] = psi_fn(ghost[(w * 2 + 0) * p.nxy + r], p.psi_kind);
            ring[(slot * 2 + 1) * T::HN + si] = psi_fn(ghost[(w * 2 + 1) * p.nxy + r], p.psi_kind);
        } else {
            float f[2 * Q];
            pull(p, S, k, z, f);
            float ra = 0.f, rb = 0.f;
#pragma unroll
            for (int i = 0; i < Q; i++) { ra += f[i]; rb += f[Q + i]; }
            ring[(slot * 2 + 0) * T::HN + si] = psi_fn(ra, p.psi_kind);
            ring[(slot * 2 + 1) * T::HN + si] = psi_fn(rb, p.psi_kind);
            if (tile && buf >= 0) {
                float* h = hold + (size_t)buf * 2 * Q * T::NI + t;
#pragma unroll
                for (int i = 0; i < 2 * Q; i++) h[i * T::NI] = f[i];
            }
        }
    };

    {
        int zb = zs - 1;
        if (!p.walls && zb < 0) zb += p.nz;
        plane(zb, 0, -1);
        plane(zs, 1, 0);
    }

    for (int z = zs; z < ze; z++) {
        const int rel = z - zs;
        int za = z + 1;
        if (!p.walls && za >= p.nz) za -= p.nz;
        plane(za, (rel + 2) & 3, (rel + 1) & 1);
        __syncthreads();
        if (!active) continue;

        const float* cur = hold + (size_t)(rel & 1) * 2 * Q * T::NI + t;
        const float* planes[3] = {ring + ((rel + 0) & 3) * 2 * T::HN, ring + ((rel + 1) & 3) * 2 * T::HN,
                                  ring + ((rel + 2) & 3) * 2 * T::HN};
        float sa[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 1; i < Q; i++) {
            const int o = si + dir_y(i) * T::HX + dir_x(i);
            const float* pl = planes[1 + dir_z(i)];
            const float qa = dir_w(i) * pl[o];
            const float qb = dir_w(i) * pl[T::HN + o];
            sa[0] += qa * dir_x(i); sa[1] += qa * dir_y(i); sa[2] += qa * dir_z(i);
            sb[0] += qb * dir_x(i); sb[1] += qb * dir_y(i); sb[2] += qb * dir_z(i);
        }
        float ra = 0.f, rb = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const float a = cur[i * T::NI], b = cur[(Q + i) * T::NI];
            const float fs = a + b;
            ra += a; rb += b;
            jx += dir_x(i) * fs; jy += dir_y(i) * fs; jz += dir_z(i) * fs;
        }
        const float pa = psi_fn(ra, p.psi_kind), pb = psi_fn(rb, p.psi_kind);
        float FA[3], FB[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            FA[d] = -pa * p.G * sb[d] + ra * p.g[d];
            FB[d] = -pb * p.G * sa[d] + rb * p.g[d];
        }
        const float rt = ra + rb;
        const float irt = 1.f / rt;
        const unsigned int n = (unsigned int)gx + (unsigned int)(gy * p.nx) + (unsigned int)z * p.nxy;
        bool hit = false;
        if (IBM) {
            hit = (__ldg(mask + (n >> 5)) >> (n & 31)) & 1u;
            if (hit) {
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const float fi = ibm_unfix(Fibm[(size_t)d * p.N + n]);
                    FA[d] += ra * irt * fi;
                    FB[d] += rb * irt * fi;
                }
            }
        }
        const float ux = jx * irt, uy = jy * irt, uz = jz * irt;
        if (!(rt > 0.f) || !(ux * ux + uy * uy + uz * uz <= 0.09f)) atomicOr(err, 1);
        const float ta = ra > 0.f ? p.tau / ra : 0.f, tb = rb > 0.f ? p.tau / rb : 0.f;
        const float uA[3] = {ux + ta * FA[0], uy + ta * FA[1], uz + ta * FA[2]};
        const float uB[3] = {ux + tb * FB[0], uy + tb * FB[1], uz + tb * FB[2]};
        const float uuA = uA[0] * uA[0] + uA[1] * uA[1] + uA[2] * uA[2];
        const float uuB = uB[0] * uB[0] + uB[1] * uB[1] + uB[2] * uB[2];
        const bool wall_next = p.walls && (z == 1 || z == p.nz - 2);
        float sA = 0.f, sB = 0.f;
        // moving directions first; the rest population closes the mass (Eq. 2, see k_bulk)
#pragma unroll
        for (int i = 1; i < Q; i++) {
            const float cuA = dir_x(i) * uA[0] + dir_y(i) * uA[1] + dir_z(i) * uA[2];
            const float cuB = dir_x(i) * uB[0] + dir_y(i) * uB[1] + dir_z(i) * uB[2];
            const float eA = dir_w(i) * ra * (1.f + 3.f * cuA + 4.5f * cuA * cuA - 1.5f * uuA);
            const float eB = dir_w(i) * rb * (1.f + 3.f * cuB + 4.5f * cuB * cuB - 1.5f * uuB);
            sA += eA;
            sB += eB;
            const float fa = cur[i * T::NI], fb = cur[(Q + i) * T::NI];
            float oA = fa + p.omega * (eA - fa);
            float oB = fb + p.omega * (eB - fb);
            unsigned int dst = n;
            int di = i;
            if (wall_next && dir_z(i) != 0 && is_wall_plane(p, z + dir_z(i))) {
                const float* U = (z + dir_z(i) == 0) ? p.ulo : p.uhi;
                const float cU = 6.f * dir_w(i) * (dir_x(i) * U[0] + dir_y(i) * U[1] + dir_z(i) * U[2]);
                oA -= cU * ra;
                oB -= cU * rb;
                dst = k.cx[1 + dir_x(i)] + k.ry[1 + dir_y(i)] + (unsigned int)(z + dir_z(i)) * p.nxy;
                di = dir_opp(i);
            }
            D[(size_t)di * p.N + dst] = oA;
            D[(size_t)(Q + di) * p.N + dst] = oB;
        }
        {
            const float fa = cur[0], fb = cur[Q * T::NI];
            D[n] = fa + p.omega * ((ra - sA) - fa);
            D[(size_t)Q * p.N + n] = fb + p.omega * ((rb - sB) - fb);
        }
        rho_out[n] = ra;
        rho_out[p.N + n] = rb;
        if (IBM && hit) {
            u_out[n] = (jx + 0.5f * (FA[0] + FB[0])) * irt;
            u_out[(size_t)p.N + n] = (jy + 0.5f * (FA[1] + FB[1])) * irt;
            u_out[(size_t)2 * p.N + n] = (jz + 0.5f * (FA[2] + FB[2])) * irt;
        }
    }
}

// ------------------------------------------------------------------------------------------------------
// Bulk kernel, row-vectorised variant (the fast path when nx is a multiple of 4; with tau != 1 nx/4 must also
// be a power of two up to 32 or a multiple of 32).
//
// A CTA owns whole x-rows: TY rows of the tile plus the rows y0-1 and y0+TY, marching through a z-segment.
// Each thread owns four consecutive nodes of a row and moves them with 16-byte loads and stores.  The pull
// of a direction with c_x = +-1 reads the aligned float4 of the source row and takes the element that
// crosses the quad boundary from the neighbouring lane with a warp shuffle; because the row (or a row
// segment of a warp) is periodic, the shuffle's wrap-around is the periodic boundary in x, and there is no
// x-halo at all.  Rows spanning several warps fetch the one missing element at a warp edge with a scalar
// load.  psi of four planes sits in a shared-memory ring ([slot][comp][row][x]).
//
// TAU1: with tau = 1 the BGK update is f* = f_eq exactly (Eq. 1), so only the five moments of a node are
// kept between planes; otherwise the populations are pulled again for the collision (an L1/L2 hit).
// ------------------------------------------------------------------------------------------------------
// MODE 0: fluid only (also with bounce-back membranes), 1: immersed-boundary force at marked nodes.  With
// bounce-back membranes every quad is stored whole, boundary nodes included: the boundary kernel, which runs
// next, rewrites every slot of a boundary node that is read later (its own rest and uncut directions; across
// a cut link the node on the other side, itself a boundary node, bounces into the slot; the slot towards a
// wall node is never read), so a uniform vector store is both correct and cheapest.  The kernel writes the
// densities of all nodes.
template <bool TAU1, int MODE, int NT, int MINB, typename T>
__global__ void __launch_bounds__(NT, MINB)
k_bulk4(LbmParams p, const T* __restrict__ S, T* __restrict__ D, float* __restrict__ rho_out,
        const float* __restrict__ ghost, const IbmF* __restrict__ Fibm, const uint32_t* __restrict__ mask,
        float* __restrict__ u_out, int* __restrict__ err, int TY) {
    constexpr bool IBM = MODE == 1;
    extern __shared__ float ring[];                      // psi [4][2][RR][nx], then moments [2][5][RR][nx]
    const int nx = p.nx;
    const int NQ = nx >> 2;
    const int RR = TY + 2;
    const int t = threadIdx.x;
    // threads past the rows (the last warp of rows whose width does not divide 32 lanes) shadow the last
    // real thread: their loads and shuffles are valid, and they write nothing
    const int nreal = NQ * RR;
    const bool phantom = t >= nreal;
    const int tr = phantom ? nreal - 1 : t;
    const int r = tr / NQ;                               // ring row: 0 <-> y0 - 1
    const int q = tr - r * NQ;
    const int x = 4 * q;
    // x-shift of the pull: rows of a power-of-two number of quads up to 32 shuffle within their own lane
    // segment (its wrap is the periodic boundary); any other row shuffles across the warp, and a lane whose
    // neighbour quad is in another warp or across the periodic wrap loads that element directly
    const bool seg_rows = NQ <= 32 && (NQ & (NQ - 1)) == 0;
    const int W = seg_rows ? NQ : 32;
    const int segl = seg_rows ? (q & (W - 1)) : (t & 31);
    const int edge = seg_rows ? 0 : (((q == 0 || (t & 31) == 0) ? 1 : 0) | ((q == NQ - 1 || (t & 31) == 31) ? 2 : 0));
    const int y0 = blockIdx.x * TY;
    const int gy = wrapi(y0 - 1 + r, p.ny);
    const bool active = !phantom && r >= 1 && r <= TY && (y0 + r - 1) < p.ny;
    const int ry[3] = {wrapi(gy - 1, p.ny) * nx, gy * nx, wrapi(gy + 1, p.ny) * nx};
    const int plane_sz = RR * nx;

    // z-segment of this CTA (uneven lengths so gridDim.y segments tile the fluid planes).  Even segments
    // march down and odd ones up, so the two CTAs sharing a segment boundary read its planes at the same
    // time (the halo plane comes from L2 instead of a second DRAM read).
    const int nzf = p.zf1 - p.zf0;
    const int zs = p.zf0 + (int)(((long long)blockIdx.y * nzf) / gridDim.y);
    const int ze = p.zf0 + (int)(((long long)(blockIdx.y + 1) * nzf) / gridDim.y);
    if (zs >= ze) return;
    const int dz = (blockIdx.y & 1) ? 1 : -1;
    const int z_first = dz > 0 ? zs : ze - 1;
    const int L = ze - zs;
    auto zwrap = [&](int z) { return p.walls ? z : (z < 0 ? z + p.nz : (z >= p.nz ? z - p.nz : z)); };

    // moments rho^A, rho^B, j of this thread's four nodes, two planes; private to the thread (no barrier)
    float* mom = ring + (size_t)8 * plane_sz + r * nx + x;
    auto mom_at = [&](int ms, int k) -> float* { return mom + (size_t)(ms * 5 + k) * plane_sz; };

    // psi of plane z into ring slot; moments into moment slot ms (if ms >= 0)
    auto plane = [&](int z, int slot, int ms) {
        float* rA = ring + (size_t)(slot * 2 + 0) * plane_sz + r * nx + x;
        float* rB = ring + (size_t)(slot * 2 + 1) * plane_sz + r * nx + x;
        if (is_wall_plane(p, z)) {
            if (phantom) return;
            const int w = z == 0 ? 0 : 1;
            const float4 ga = *reinterpret_cast<const float4*>(ghost + (w * 2 + 0) * p.nxy + gy * nx + x);
            const float4 gb = *reinterpret_cast<const float4*>(ghost + (w * 2 + 1) * p.nxy + gy * nx + x);
            *reinterpret_cast<float4*>(rA) = make_float4(psi_fn(ga.x, p.psi_kind), psi_fn(ga.y, p.psi_kind),
                                                         psi_fn(ga.z, p.psi_kind), psi_fn(ga.w, p.psi_kind));
            *reinterpret_cast<float4*>(rB) = make_float4(psi_fn(gb.x, p.psi_kind), psi_fn(gb.y, p.psi_kind),
                                                         psi_fn(gb.z, p.psi_kind), psi_fn(gb.w, p.psi_kind));
            return;
        }
        Mom4 m;
#pragma unroll
        for (int k = 0; k < 4; k++) m.ra[k] = m.rb[k] = m.jx[k] = m.jy[k] = m.jz[k] = 0.f;
        const PullCtx pc = pull_ctx(p, ry, z);
        pull_all(p, S, pc, x, segl, W, edge, m, AllDirs{});
        if (phantom) return;                             // its pulls only fed the shuffles
        *reinterpret_cast<float4*>(rA) = make_float4(psi_fn(m.ra[0], p.psi_kind), psi_fn(m.ra[1], p.psi_kind),
                                                     psi_fn(m.ra[2], p.psi_kind), psi_fn(m.ra[3], p.psi_kind));
        *reinterpret_cast<float4*>(rB) = make_float4(psi_fn(m.rb[0], p.psi_kind), psi_fn(m.rb[1], p.psi_kind),
                                                     psi_fn(m.rb[2], p.psi_kind), psi_fn(m.rb[3], p.psi_kind));
        if (ms >= 0) {
            *reinterpret_cast<float4*>(mom_at(ms, 0)) = make_float4(m.ra[0], m.ra[1], m.ra[2], m.ra[3]);
            *reinterpret_cast<float4*>(mom_at(ms, 1)) = make_float4(m.rb[0], m.rb[1], m.rb[2], m.rb[3]);
            *reinterpret_cast<float4*>(mom_at(ms, 2)) = make_float4(m.jx[0], m.jx[1], m.jx[2], m.jx[3]);
            *reinterpret_cast<float4*>(mom_at(ms, 3)) = make_float4(m.jy[0], m.jy[1], m.jy[2], m.jy[3]);
            *reinterpret_cast<float4*>(mom_at(ms, 4)) = make_float4(m.jz[0], m.jz[1], m.jz[2], m.jz[3]);
        }
    };

    plane(zwrap(z_first - dz), 0, -1);
    plane(z_first, 1, 0);

    for (int rel = 0; rel < L; rel++) {
        const int z = z_first + rel * dz;
        plane(zwrap(z + dz), (rel + 2) & 3, (rel + 1) & 1);
        __syncthreads();
        // lanes of this warp that collide (whole row segments share `active`, so shuffles stay within them)
        const unsigned int lanes = __ballot_sync(0xffffffffu, active);

        if (active) {
            // ---- Shan-Chen force (Eq. 13) for the four nodes from the psi ring
            float sa[3][4], sb[3][4];                   // sum_i w_i psi^A(x+c_i) c_i, same with psi^B
#pragma unroll
            for (int d = 0; d < 3; d++)
#pragma unroll
                for (int k = 0; k < 4; k++) sa[d][k] = sb[d][k] = 0.f;
            // ring slots of the planes z - 1, z, z + 1 (the march direction decides which one is ahead)
            const int s_back = rel & 3, s_ahead = (rel + 2) & 3;
            const float* slots[3] = {ring + (size_t)(dz > 0 ? s_back : s_ahead) * 2 * plane_sz,
                                     ring + (size_t)((rel + 1) & 3) * 2 * plane_sz,
                                     ring + (size_t)(dz > 0 ? s_ahead : s_back) * 2 * plane_sz};
#pragma unroll
            for (int cz = -1; cz <= 1; cz++)
#pragma unroll
                for (int cy = -1; cy <= 1; cy++) {
                    if (cy != 0 && cz != 0) {
                        // corner rows: only c_x = 0 (directions 15-18)
                        const float w = 1.f / 36.f;
#pragma unroll
                        for (int c = 0; c < 2; c++) {
                            const float4 v = *reinterpret_cast<const float4*>(slots[1 + cz] + c * plane_sz +
                                                                              (r + cy) * nx + x);
                            const float V[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int k = 0; k < 4; k++) {
                                if (c == 0) { sa[1][k] += w * cy * V[k]; sa[2][k] += w * cz * V[k]; }
                                else { sb[1][k] += w * cy * V[k]; sb[2][k] += w * cz * V[k]; }
                            }
                        }
                        continue;
                    }
                    const bool centre = cy == 0 && cz == 0;
                    const float wc = centre ? 0.f : 1.f / 18.f;        // c_x = 0 neighbour (x, y+cy, z+cz)
                    const float wx = centre ? 1.f / 18.f : 1.f / 36.f; // c_x = +-1 neighbours
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        float w6[6];
                        window6(slots[1 + cz] + c * plane_sz + (r + cy) * nx, x, nx, w6);
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            const float vm = w6[k], v0 = w6[k + 1], vp = w6[k + 2];   // x-1, x, x+1
                            const float fx = wx * (vp - vm);
                            const float sum3 = wx * (vp + vm) + wc * v0;
                            if (c == 0) {
                                sa[0][k] += fx; sa[1][k] += cy * sum3; sa[2][k] += cz * sum3;
                            } else {
                                sb[0][k] += fx; sb[1][k] += cy * sum3; sb[2][k] += cz * sum3;
                            }
                        }
                    }
                }

            const unsigned int n0 = (unsigned)x + (unsigned)gy * nx + (unsigned)z * p.nxy;
            uint32_t bits = 0;
            if (IBM) bits = (__ldg(mask + (n0 >> 5)) >> (n0 & 31)) & 0xFu;
            float uA[4][3], uB[4][3], ra[4], rb[4], jxa[4], jya[4], jza[4];
            {
                const int ms = rel & 1;
                const float4 a = *reinterpret_cast<const float4*>(mom_at(ms, 0));
                const float4 b = *reinterpret_cast<const float4*>(mom_at(ms, 1));
                const float4 jx4 = *reinterpret_cast<const float4*>(mom_at(ms, 2));
                const float4 jy4 = *reinterpret_cast<const float4*>(mom_at(ms, 3));
                const float4 jz4 = *reinterpret_cast<const float4*>(mom_at(ms, 4));
                ra[0] = a.x; ra[1] = a.y; ra[2] = a.z; ra[3] = a.w;
                rb[0] = b.x; rb[1] = b.y; rb[2] = b.z; rb[3] = b.w;
                jxa[0] = jx4.x; jxa[1] = jx4.y; jxa[2] = jx4.z; jxa[3] = jx4.w;
                jya[0] = jy4.x; jya[1] = jy4.y; jya[2] = jy4.z; jya[3] = jy4.w;
                jza[0] = jz4.x; jza[1] = jz4.y; jza[2] = jz4.z; jza[3] = jz4.w;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float pa = psi_fn(ra[k], p.psi_kind), pb = psi_fn(rb[k], p.psi_kind);
                const float rt = ra[k] + rb[k];
                const float irt = 1.f / rt;
                float FA[3], FB[3];
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    FA[d] = -pa * p.G * sb[d][k] + ra[k] * p.g[d];
                    FB[d] = -pb * p.G * sa[d][k] + rb[k] * p.g[d];
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
                uA[k][0] = ux + ta * FA[0]; uA[k][1] = uy + ta * FA[1]; uA[k][2] = uz + ta * FA[2];
                uB[k][0] = ux + tb * FB[0]; uB[k][1] = uy + tb * FB[1]; uB[k][2] = uz + tb * FB[2];
                if (IBM && ((bits >> k) & 1u)) {
                    // half-force velocity (Eq. 5) for the immersed-boundary interpolation
                    u_out[n0 + k] = (jxa[k] + 0.5f * (FA[0] + FB[0])) * irt;
                    u_out[(size_t)p.N + n0 + k] = (jya[k] + 0.5f * (FA[1] + FB[1])) * irt;
                    u_out[(size_t)2 * p.N + n0 + k] = (jza[k] + 0.5f * (FA[2] + FB[2])) * irt;
                }
            }
            // ---- equilibrium (Eq. 2) and BGK update, direction by direction, float4 stores
            const bool wall_next = p.walls && (z == 1 || z == p.nz - 2);
            float uuA[4], uuB[4], sA[4], sB[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                uuA[k] = uA[k][0] * uA[k][0] + uA[k][1] * uA[k][1] + uA[k][2] * uA[k][2];
                uuB[k] = uB[k][0] * uB[k][0] + uB[k][1] * uB[k][1] + uB[k][2] * uB[k][2];
                sA[k] = sB[k] = 0.f;
            }
            PullCtx pc;
            if (!TAU1) pc = pull_ctx(p, ry, z);
            auto emit = [&](auto Ic) {
                constexpr int I = decltype(Ic)::value;
                float oA[4], oB[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    float eA, eB;
                    if (I == 0) {
                        eA = ra[k] - sA[k];
                        eB = rb[k] - sB[k];
                        if (TAU1 && sizeof(T) == 2) {   // unbiased rounding of the mass-closing value
                            const uint32_t h = dither_bits(n0 + k, ra[k], rb[k]);
                            eA = pdither(eA, h >> 16, D);
                            eB = pdither(eB, h & 0xffffu, D);
                        }
                    } else {
                        const float cuA = dir_x(I) * uA[k][0] + dir_y(I) * uA[k][1] + dir_z(I) * uA[k][2];
                        const float cuB = dir_x(I) * uB[k][0] + dir_y(I) * uB[k][1] + dir_z(I) * uB[k][2];
                        eA = dir_w(I) * ra[k] * (1.f + 3.f * cuA + 4.5f * cuA * cuA - 1.5f * uuA[k]);
                        eB = dir_w(I) * rb[k] * (1.f + 3.f * cuB + 4.5f * cuB * cuB - 1.5f * uuB[k]);
                        if (TAU1) {             // the values as stored (exact for FP32)
                            eA = pround(eA, D);
                            eB = pround(eB, D);
                        }
                        sA[k] += eA;
                        sB[k] += eB;
                    }
                    oA[k] = eA;
                    oB[k] = eB;
                }
                if (!TAU1) {
                    const float4 fa = pull_comp<I, T>(p, S, pc, x, segl, W, edge, lanes);
                    const float4 fb = pull_comp<I, T>(p, S + (size_t)Q * p.N, pc, x, segl, W, edge, lanes);
                    const float FA4[4] = {fa.x, fa.y, fa.z, fa.w}, FB4[4] = {fb.x, fb.y, fb.z, fb.w};
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        oA[k] = FA4[k] + p.omega * (oA[k] - FA4[k]);
                        oB[k] = FB4[k] + p.omega * (oB[k] - FB4[k]);
                    }
                }
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
            // moving directions first, the rest population last (it closes the mass, see k_bulk)
            emit(std::integral_constant<int, 1>{});  emit(std::integral_constant<int, 2>{});
            emit(std::integral_constant<int, 3>{});  emit(std::integral_constant<int, 4>{});
            emit(std::integral_constant<int, 5>{});  emit(std::integral_constant<int, 6>{});
            emit(std::integral_constant<int, 7>{});  emit(std::integral_constant<int, 8>{});
            emit(std::integral_constant<int, 9>{});  emit(std::integral_constant<int, 10>{});
            emit(std::integral_constant<int, 11>{}); emit(std::integral_constant<int, 12>{});
            emit(std::integral_constant<int, 13>{}); emit(std::integral_constant<int, 14>{});
            emit(std::integral_constant<int, 15>{}); emit(std::integral_constant<int, 16>{});
            emit(std::integral_constant<int, 17>{}); emit(std::integral_constant<int, 18>{});
            emit(std::integral_constant<int, 0>{});
            *reinterpret_cast<float4*>(rho_out + n0) = make_float4(ra[0], ra[1], ra[2], ra[3]);
            *reinterpret_cast<float4*>(rho_out + p.N + n0) = make_float4(rb[0], rb[1], rb[2], rb[3]);
        }
    }
}

// Tile height (rows per CTA) of the row-vectorised kernel with nthreads threads, or 0 if it does not fit.
static int bulk4_rows(const LbmParams& p, int nthreads) {
    if (p.nx % 4) return 0;
    const int NQ = p.nx / 4;
    const bool pow2 = (NQ & (NQ - 1)) == 0;
    const bool aligned = (NQ <= 32 && pow2) || NQ % 32 == 0;
    // rows of any other width shuffle across whole warps, which the collision's re-pull of tau != 1 (with
    // only the colliding rows' lanes) cannot do
    if (!aligned && p.omega != 1.0f) return 0;
    if (NQ > nthreads / 3) return 0;                   // need at least one tile row plus two halo rows
    int RR = nthreads / NQ;
    if (aligned) {
        while (RR > 3 && (RR * NQ) % 32) RR--;
        if ((RR * NQ) % 32) return 0;
    } else {
        while (RR > 3 && (RR * NQ + 31) / 32 * 32 > nthreads) RR--;    // the last warp may carry phantoms
    }
    int TY = RR - 2;
    if (TY > p.ny) TY = p.ny;
    return TY;
}

constexpr int BTX = 32, BTY = 8;

// SCBB_BULK_VARIANT: unset -> the two-kernel bulk phase wherever it applies (tau = 1), else the fused
// row-vectorised kernel (nx a multiple of 4), else the general fused kernel; "4": the fused kernels only;
// "2": the general fused kernel only.  Results agree to rounding (each path is tested against the oracle).
int bulk_variant() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("SCBB_BULK_VARIANT");
        v = (e && (e[0] == '2' || e[0] == '4') && e[1] == 0) ? e[0] - '0' : 5;
    }
    return v;
}

static void bulk_geometry(const LbmParams& p, dim3& grid, int& threads) {
    int nzf = p.zf1 - p.zf0;
    grid = dim3((p.nx + BTX - 1) / BTX, (p.ny + BTY - 1) / BTY, (nzf + p.lz - 1) / p.lz);
    threads = Tile<BTX, BTY>::HN;
}

// Row-vectorised geometry: TY tile rows (+2 halo rows) per CTA of nthreads threads, z split into
// segments of at least min_planes planes so that the grid fills the 152 SMs (cps CTAs resident per SM) in as
// few waves as possible.
static bool bulk4_geometry(const LbmParams& p, int nthreads, int cps, int min_planes, LbmParams& q, dim3& grid,
                           int& threads, int& TY, size_t& smem) {
    TY = bulk4_rows(p, nthreads);
    if (TY <= 0) return false;
    const int NQ = p.nx / 4;
    const bool aligned = (NQ <= 32 && (NQ & (NQ - 1)) == 0) || NQ % 32 == 0;
    if (aligned) {
        while ((NQ * (TY + 2)) % 32) TY++;
        threads = NQ * (TY + 2);
    } else {
        threads = (NQ * (TY + 2) + 31) / 32 * 32;     // rows, then phantom threads up to a whole warp
    }
    if (threads > nthreads) return false;
    const int cols = (p.ny + TY - 1) / TY;
    const int nzf = p.zf1 - p.zf0;
    const int slots = 152 * cps;
    int nseg = 1;
    double best = -1.0;
    for (int w = 1; w <= 4; w++) {
        int ns = (slots * w) / cols;
        if (ns < 1) ns = 1;
        if (ns > nzf / min_planes) ns = nzf / min_planes > 0 ? nzf / min_planes : 1;
        const int nb = cols * ns;
        const int waves = (nb + slots - 1) / slots;
        const double eff = (double)nb / ((double)slots * waves) - 0.02 * waves;
        if (eff > best + 1e-9) { best = eff; nseg = ns; }
    }
    q = p;
    q.lz = (nzf + nseg - 1) / nseg;
    grid = dim3(cols, nseg, 1);
    smem = (size_t)(4 * 2 + 2 * 5) * (TY + 2) * p.nx * sizeof(float);
    return true;
}

template <bool TAU1, int MODE, int NT, int MINB, typename T>
static void launch_b4t(const LbmParams& q, dim3 grid, int threads, size_t smem, int TY, const T* S, T* D,
                       float* rho, const float* ghost, const IbmF* Fibm, const uint32_t* mask, float* u, int* err,
                       cudaStream_t st) {
    static size_t attr = 0;
    if (smem > attr) {
        cudaFuncSetAttribute(k_bulk4<TAU1, MODE, NT, MINB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr = smem;
    }
    k_bulk4<TAU1, MODE, NT, MINB, T><<<grid, threads, smem, st>>>(q, S, D, rho, ghost, Fibm, mask, u, err, TY);
}

// S, D point to populations of the type q.store names
template <bool TAU1, int MODE, int NT, int MINB>
static void launch_b4(const LbmParams& q, dim3 grid, int threads, size_t smem, int TY, const float* S, float* D,
                      float* rho, const float* ghost, const IbmF* Fibm, const uint32_t* mask, float* u, int* err,
                      cudaStream_t st) {
    with_plain_storage(q.store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        launch_b4t<TAU1, MODE, NT, MINB, T>(q, grid, threads, smem, TY, reinterpret_cast<const T*>(S),
                                            reinterpret_cast<T*>(D), rho, ghost, Fibm, mask, u, err, st);
    });
}

template <int NT, int MINB>
static bool try_b4(const LbmParams& p, int min_planes, const float* S, float* D, float* rho, const float* ghost,
                   const IbmF* Fibm, const uint32_t* mask, float* u, int* err, int mode, cudaStream_t st,
                   int* blocks) {
    LbmParams q;
    dim3 grid;
    int threads, TY;
    size_t smem;
    if (!bulk4_geometry(p, NT, MINB, min_planes, q, grid, threads, TY, smem)) return false;
    if (blocks) {
        *blocks = (int)(grid.x * grid.y);
        return true;
    }
    const bool tau1 = p.omega == 1.0f;
#define B4_ARGS q, grid, threads, smem, TY, S, D, rho, ghost, Fibm, mask, u, err, st
    if (tau1) {
        if (mode == 1) launch_b4<true, 1, NT, MINB>(B4_ARGS);
        else launch_b4<true, 0, NT, MINB>(B4_ARGS);
    } else {
        if (mode == 1) launch_b4<false, 1, NT, MINB>(B4_ARGS);
        else launch_b4<false, 0, NT, MINB>(B4_ARGS);
    }
#undef B4_ARGS
    return true;
}

static bool dispatch_b4(const LbmParams& p, const float* S, float* D, float* rho, const float* ghost,
                        const IbmF* Fibm, const uint32_t* mask, float* u, int* err, int mode,
                        cudaStream_t st, int* blocks) {
    switch (p.b4cfg) {
        case 1: return try_b4<256, 2>(p, 6, S, D, rho, ghost, Fibm, mask, u, err, mode, st, blocks);
        case 2: return try_b4<512, 1>(p, 3, S, D, rho, ghost, Fibm, mask, u, err, mode, st, blocks);
        case 3: return try_b4<256, 2>(p, 3, S, D, rho, ghost, Fibm, mask, u, err, mode, st, blocks);
        default: return try_b4<512, 1>(p, 6, S, D, rho, ghost, Fibm, mask, u, err, mode, st, blocks);
    }
}

bool bulk_vectorised(const LbmParams& p) {
    if (bulk_split(p)) return true;
    int nb = 0;
    return bulk_variant() >= 4 && dispatch_b4(p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                              nullptr, 0, 0, &nb);
}

bool bulk_writes_ghost(const LbmParams& p) { return bulk_split(p); }

int bulk_grid_blocks(const LbmParams& p) {
    int nb = 0;
    if (bulk_split(p)) return split_grid_blocks(p);
    if (bulk_variant() >= 4 && dispatch_b4(p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                           0, 0, &nb))
        return nb;
    dim3 g;
    int th;
    bulk_geometry(p, g, th);
    return (int)(g.x * g.y * g.z);
}

void launch_bulk(const LbmParams& p, const float* S, float* D, float* rho, float* J, float* ghost, const IbmF* Fibm,
                 const uint32_t* mask, float* u, int* err, int mode, cudaStream_t st) {
    const bool ibm = mode == 1;
    if (J && bulk_split(p)) {
        launch_split(p, S, D, rho, J, ghost, Fibm, mask, u, err, mode, st);
        return;
    }
    if (bulk_variant() >= 4 && dispatch_b4(p, S, D, rho, ghost, Fibm, mask, u, err, mode, st, nullptr)) return;
    dim3 grid;
    int threads;
    bulk_geometry(p, grid, threads);
    constexpr int sm = bulk2_smem_bytes<BTX, BTY>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_bulk2<BTX, BTY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        cudaFuncSetAttribute(k_bulk2<BTX, BTY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        attr = true;
    }
    if (ibm)
        k_bulk2<BTX, BTY, true><<<grid, threads, sm, st>>>(p, S, D, rho, ghost, Fibm, mask, u, err);
    else
        k_bulk2<BTX, BTY, false><<<grid, threads, sm, st>>>(p, S, D, rho, ghost, Fibm, mask, u, err);
}

void launch_init_state(const LbmParams& p, float* S, const float* rho_st, const float* u_st, cudaStream_t st) {
    with_storage(p.store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        k_init_state<T, float><<<(p.N + 255) / 256, 256, 0, st>>>(p, reinterpret_cast<T*>(S), rho_st, u_st);
    });
}

void launch_init_state(const LbmParams& p, float* S, const double* rho_st, const double* u_st, cudaStream_t st) {
    with_storage(p.store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        k_init_state<T, double><<<(p.N + 255) / 256, 256, 0, st>>>(p, reinterpret_cast<T*>(S), rho_st, u_st);
    });
}

void launch_wall_ghost(const LbmParams& p, const float* S, float* wall_rho, float* ghost, cudaStream_t st) {
    with_plain_storage(p.store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        k_wall_planes_rho<T><<<(2 * p.nxy + 255) / 256, 256, 0, st>>>(p, reinterpret_cast<const T*>(S), wall_rho);
    });
    k_wall_ghost<<<(4 * p.nxy + 255) / 256, 256, 0, st>>>(p, wall_rho, ghost);
}

// ------------------------------------------------------------------------------------------------------
// Exports of the current state.  what = 0: rho^A, rho^B, u (5 N floats); what = 1: populations in the
// [c][node][i] order (38 N floats).  Wall nodes report 0.
// ------------------------------------------------------------------------------------------------------
// what = 2, 3: the populations of component A or B only, [node][i] (19 N floats)
template <typename T>
__global__ void k_export(LbmParams p, const T* __restrict__ S, float* __restrict__ out, int what,
                         double* __restrict__ out64) {
    unsigned int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    int z = n / p.nxy;
    int r = n - z * p.nxy;
    int y = r / p.nx, x = r - y * p.nx;
    float f[2 * Q];
    if (is_wall_plane(p, z)) {
#pragma unroll
        for (int i = 0; i < 2 * Q; i++) f[i] = 0.f;
    } else {
        Cols k;
        k.cx[0] = wrapi(x - 1, p.nx); k.cx[1] = x; k.cx[2] = wrapi(x + 1, p.nx);
        k.ry[0] = wrapi(y - 1, p.ny) * p.nx; k.ry[1] = y * p.nx; k.ry[2] = wrapi(y + 1, p.ny) * p.nx;
        pull(p, S, k, z, f);
        if (is_onsite_plane(p, z)) onsite_fix(p, z, f);
    }
    if (what == 1) {
#pragma unroll
        for (int i = 0; i < Q; i++) {
            out[(size_t)n * Q + i] = f[i];
            out[(size_t)(p.N + n) * Q + i] = f[Q + i];
        }
        return;
    }
    if (what == 2 || what == 3) {
        const int c = what - 2;
#pragma unroll
        for (int i = 0; i < Q; i++) out[(size_t)n * Q + i] = f[c * Q + i];
        return;
    }
    if (what >= 16) {                                  // one direction of one component: f[c Q + i], c Q + i = what - 16
        const int ci = what - 16;
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < 2 * Q; k++)
            if (k == ci) v = f[k];
        out[n] = v;
        return;
    }
    // read-out in FP64: the momentum is a sum of populations with +- cancellations, whose FP32 rounding
    // (about 19 * 2^-24 of the largest population) would otherwise show in the exported velocity
    double ra = 0.0, rb = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        ra += f[i]; rb += f[Q + i];
        const double fs = (double)f[i] + (double)f[Q + i];
        jx += dir_x(i) * fs; jy += dir_y(i) * fs; jz += dir_z(i) * fs;
    }
    const double rt = ra + rb;
    const double irt = rt > 0.0 ? 1.0 / rt : 0.0;
    if (what == 4) {                                   // the same FP32 values, widened to FP64
        out64[n] = (double)(float)ra;
        out64[p.N + n] = (double)(float)rb;
        out64[2 * (size_t)p.N + n] = (double)(float)(jx * irt);
        out64[3 * (size_t)p.N + n] = (double)(float)(jy * irt);
        out64[4 * (size_t)p.N + n] = (double)(float)(jz * irt);
        return;
    }
    out[n] = (float)ra;
    out[p.N + n] = (float)rb;
    out[2 * (size_t)p.N + n] = (float)(jx * irt);
    out[3 * (size_t)p.N + n] = (float)(jy * irt);
    out[4 * (size_t)p.N + n] = (float)(jz * irt);
}

void launch_export(const LbmParams& p, const float* S, float* out, int what, cudaStream_t st, double* out64) {
    with_storage(p.store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        k_export<T><<<(p.N + 255) / 256, 256, 0, st>>>(p, reinterpret_cast<const T*>(S), out, what, out64);
    });
}

// ------------------------------------------------------------------------------------------------------
// FP64 reductions of the current state: mass per component and total momentum (fixed order: per-block
// partials, then one block sums them), red[0..4] = M^A, M^B, P_x, P_y, P_z.
// ------------------------------------------------------------------------------------------------------
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 1024;

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_moments_partial(LbmParams p, const T* __restrict__ S,
                                                                 double* __restrict__ part) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (unsigned int n = blockIdx.x * blockDim.x + threadIdx.x; n < p.N; n += gridDim.x * blockDim.x) {
        int z = n / p.nxy;
        if (is_wall_plane(p, z)) continue;
        int r = n - z * p.nxy;
        int y = r / p.nx, x = r - y * p.nx;
        Cols k;
        k.cx[0] = wrapi(x - 1, p.nx); k.cx[1] = x; k.cx[2] = wrapi(x + 1, p.nx);
        k.ry[0] = wrapi(y - 1, p.ny) * p.nx; k.ry[1] = y * p.nx; k.ry[2] = wrapi(y + 1, p.ny) * p.nx;
        float f[2 * Q];
        pull(p, S, k, z, f);
        if (is_onsite_plane(p, z)) onsite_fix(p, z, f);
        for (int i = 0; i < Q; i++) {
            double a = f[i], b = f[Q + i];
            acc[0] += a; acc[1] += b;
            acc[2] += dir_x(i) * (a + b); acc[3] += dir_y(i) * (a + b); acc[4] += dir_z(i) * (a + b);
        }
    }
    __shared__ double sh[5][RED_THREADS];
    for (int q = 0; q < 5; q++) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 5; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; q++) part[blockIdx.x * 5 + q] = sh[q][0];
}

__global__ void __launch_bounds__(RED_THREADS) k_sum_partials(const double* __restrict__ part, int nb, int nq,
                                                              double* __restrict__ out) {
    __shared__ double sh[RED_THREADS];
    for (int q = 0; q < nq; q++) {
        double a = 0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) a += part[b * nq + q];
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = sh[0];
        __syncthreads();
    }
}

void launch_moments_reduce(const LbmParams& p, const float* S, double* red, cudaStream_t st) {
    // red must hold 8 + 5 * RED_BLOCKS doubles; result in red[0..4]
    with_storage(p.store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        k_moments_partial<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(p, reinterpret_cast<const T*>(S), red + 8);
    });
    k_sum_partials<<<1, RED_THREADS, 0, st>>>(red + 8, RED_BLOCKS, 5, red);
}

}  // namespace scbb
