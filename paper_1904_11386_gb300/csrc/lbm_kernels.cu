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

#include "scbb_internal.cuh"

namespace scbb {

__device__ __forceinline__ int wrapi(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

__device__ __forceinline__ float psi_fn(float rho, int kind) {
    // psi = 1 - exp(-rho/rho0) with rho0 = 1 (Sec. II.D), or psi = rho
    return kind == 1 ? rho : -expm1f(-rho);
}

__device__ __forceinline__ bool is_wall_plane(const LbmParams& p, int z) {
    return p.walls && (z == 0 || z == p.nz - 1);
}

// ------------------------------------------------------------------------------------------------------
// Initial state: slot (c, i, y) holds the population that node x = y + c_i pulls, f_eq,i(rho^c(x), u(x)).
// ------------------------------------------------------------------------------------------------------
__global__ void k_init_state(LbmParams p, float* __restrict__ S, const float* __restrict__ rho_st,
                             const float* __restrict__ u_st) {
    unsigned int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    int z = n / p.nxy;
    int r = n - z * p.nxy;
    int y = r / p.nx, x = r - y * p.nx;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        int zz = z + dir_z(i);
        float v0 = 0.f, v1 = 0.f;
        bool ok = true;
        if (p.walls) ok = (zz >= 1 && zz <= p.nz - 2);
        else zz = wrapi(zz, p.nz);
        if (ok) {
            unsigned int m = wrapi(x + dir_x(i), p.nx) + p.nx * (wrapi(y + dir_y(i), p.ny) + p.ny * zz);
            float ux = u_st[m], uy = u_st[p.N + m], uz = u_st[2 * p.N + m];
            float cu = dir_x(i) * ux + dir_y(i) * uy + dir_z(i) * uz;
            float uu = ux * ux + uy * uy + uz * uz;
            float e = dir_w(i) * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * uu);
            v0 = e * rho_st[m];
            v1 = e * rho_st[p.N + m];
        }
        S[(size_t)i * p.N + n] = v0;
        S[(size_t)(Q + i) * p.N + n] = v1;
    }
}

// ------------------------------------------------------------------------------------------------------
// Pull helper: populations arriving at (gx, gy, z) from its 18 neighbours (x, y periodic).
// ------------------------------------------------------------------------------------------------------
struct Cols {
    int cx[3];          // x - 1, x, x + 1 (wrapped)
    int ry[3];          // (y - 1) nx, y nx, (y + 1) nx (wrapped)
};

__device__ __forceinline__ void pull(const LbmParams& p, const float* __restrict__ S, const Cols& k, int z,
                                     float (&f)[2 * Q]) {
    int zm = z - 1, zp = z + 1;
    if (!p.walls) {
        zm = zm < 0 ? zm + p.nz : zm;
        zp = zp >= p.nz ? zp - p.nz : zp;
    }
    const int pz[3] = {zm * p.nxy, z * p.nxy, zp * p.nxy};
#pragma unroll
    for (int i = 0; i < Q; i++) {
        // source node x - c_i
        unsigned int m = k.cx[1 - dir_x(i)] + k.ry[1 - dir_y(i)] + pz[1 - dir_z(i)];
        f[i] = __ldg(S + (size_t)i * p.N + m);
        f[Q + i] = __ldg(S + (size_t)(Q + i) * p.N + m);
    }
}

// ------------------------------------------------------------------------------------------------------
// Virtual densities of the wall planes (neutral wetting): the wall node (x, y, 0) is seen with the mean
// density of its five fluid neighbours (x, y, 1), (x +- 1, y, 1), (x, y +- 1, 1); likewise at the top.
// ------------------------------------------------------------------------------------------------------
__global__ void k_wall_planes_rho(LbmParams p, const float* __restrict__ S, float* __restrict__ wall_rho) {
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

// ------------------------------------------------------------------------------------------------------
// Bulk kernel.  Block = (TX+2)(TY+2) threads: TX*TY tile nodes first, then the halo ring.
// ------------------------------------------------------------------------------------------------------
template <int TX, int TY>
struct Tile {
    static constexpr int HX = TX + 2, HY = TY + 2, HN = HX * HY, NI = TX * TY;
};

template <int TX, int TY, bool IBM>
__global__ void __launch_bounds__(Tile<TX, TY>::HN)
k_bulk(LbmParams p, const float* __restrict__ S, float* __restrict__ D, float* __restrict__ rho_out,
       const float* __restrict__ ghost, const float* __restrict__ Fibm, const uint32_t* __restrict__ mask,
       float* __restrict__ u_out, int* __restrict__ err) {
    using T = Tile<TX, TY>;
    __shared__ float sp[4][2][T::HN];        // psi^A, psi^B of four consecutive planes (ring)

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
    const bool active = (t < T::NI) && (x0 + lx < p.nx) && (y0 + ly < p.ny);
    const int si = (ly + 1) * T::HX + (lx + 1);

    Cols k;
    k.cx[0] = wrapi(gx - 1, p.nx); k.cx[1] = gx; k.cx[2] = wrapi(gx + 1, p.nx);
    k.ry[0] = wrapi(gy - 1, p.ny) * p.nx; k.ry[1] = gy * p.nx; k.ry[2] = wrapi(gy + 1, p.ny) * p.nx;

    const int zs = p.zf0 + blockIdx.z * p.lz;
    const int ze = min(zs + p.lz, p.zf1);
    if (zs >= ze) return;                    // uniform over the block

    float cur[2 * Q], nxt[2 * Q];

    // psi of plane z into ring slot `slot`; pulled populations land in f
    auto plane = [&](int z, int slot, float (&f)[2 * Q]) {
        if (is_wall_plane(p, z)) {
            const int w = z == 0 ? 0 : 1;
            const int r = gx + gy * p.nx;
            sp[slot][0][si] = psi_fn(ghost[(w * 2 + 0) * p.nxy + r], p.psi_kind);
            sp[slot][1][si] = psi_fn(ghost[(w * 2 + 1) * p.nxy + r], p.psi_kind);
        } else {
            pull(p, S, k, z, f);
            float ra = 0.f, rb = 0.f;
#pragma unroll
            for (int i = 0; i < Q; i++) { ra += f[i]; rb += f[Q + i]; }
            sp[slot][0][si] = psi_fn(ra, p.psi_kind);
            sp[slot][1][si] = psi_fn(rb, p.psi_kind);
        }
    };

    {
        int zb = zs - 1;
        if (!p.walls && zb < 0) zb += p.nz;
        plane(zb, 0, nxt);                   // nxt is scratch here
        plane(zs, 1, cur);
    }

    for (int z = zs; z < ze; z++) {
        const int rel = z - zs;
        int za = z + 1;
        if (!p.walls && za >= p.nz) za -= p.nz;
        plane(za, (rel + 2) & 3, nxt);
        __syncthreads();

        if (active) {
            const float* pm = sp[(rel + 0) & 3][0];   // plane z - 1
            const float* p0 = sp[(rel + 1) & 3][0];   // plane z
            const float* pp = sp[(rel + 2) & 3][0];   // plane z + 1
            const float* planes[3] = {pm, p0, pp};
            // Shan-Chen force (Eq. 13): F^A = -psi^A G sum_i w_i psi^B(x + c_i) c_i, and the mirror for B
            float sa[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 1; i < Q; i++) {
                const int o = si + dir_y(i) * T::HX + dir_x(i);
                const float* pl = planes[1 + dir_z(i)];
                // ring slots store psi^A then psi^B, T::HN floats apart
                const float qa = dir_w(i) * pl[o];
                const float qb = dir_w(i) * pl[T::HN + o];
                sa[0] += qa * dir_x(i); sa[1] += qa * dir_y(i); sa[2] += qa * dir_z(i);
                sb[0] += qb * dir_x(i); sb[1] += qb * dir_y(i); sb[2] += qb * dir_z(i);
            }
            float ra = 0.f, rb = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const float fs = cur[i] + cur[Q + i];
                ra += cur[i];
                rb += cur[Q + i];
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
                    // immersed-boundary force density, shared by the components in proportion to rho^c
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        const float fi = Fibm[(size_t)d * p.N + n];
                        FA[d] += ra * irt * fi;
                        FB[d] += rb * irt * fi;
                    }
                }
            }
            const float ux = jx * irt, uy = jy * irt, uz = jz * irt;   // common velocity u'
            if (!(rt > 0.f) || ux * ux + uy * uy + uz * uz > 0.01f) atomicOr(err, 1);
            const float ta = ra > 0.f ? p.tau / ra : 0.f, tb = rb > 0.f ? p.tau / rb : 0.f;
            const float uA[3] = {ux + ta * FA[0], uy + ta * FA[1], uz + ta * FA[2]};
            const float uB[3] = {ux + tb * FB[0], uy + tb * FB[1], uz + tb * FB[2]};
            const float uuA = uA[0] * uA[0] + uA[1] * uA[1] + uA[2] * uA[2];
            const float uuB = uB[0] * uB[0] + uB[1] * uB[1] + uB[2] * uB[2];
            const bool wall_next = p.walls && (z == 1 || z == p.nz - 2);
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const float cuA = dir_x(i) * uA[0] + dir_y(i) * uA[1] + dir_z(i) * uA[2];
                const float cuB = dir_x(i) * uB[0] + dir_y(i) * uB[1] + dir_z(i) * uB[2];
                const float eA = dir_w(i) * ra * (1.f + 3.f * cuA + 4.5f * cuA * cuA - 1.5f * uuA);
                const float eB = dir_w(i) * rb * (1.f + 3.f * cuB + 4.5f * cuB * cuB - 1.5f * uuB);
                float oA = cur[i] + p.omega * (eA - cur[i]);
                float oB = cur[Q + i] + p.omega * (eB - cur[Q + i]);
                unsigned int dst = n;
                int di = i;
                if (wall_next && dir_z(i) != 0 && is_wall_plane(p, z + dir_z(i))) {
                    // half-way bounce-back on a moving wall (Eq. 11, v0 = wall velocity): the population leaving
                    // along c_i returns along -c_i; it is stored where this node pulls direction opp(i) from
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
            rho_out[n] = ra;
            rho_out[p.N + n] = rb;
            if (IBM && hit) {
                u_out[n] = (jx + 0.5f * (FA[0] + FB[0])) * irt;
                u_out[(size_t)p.N + n] = (jy + 0.5f * (FA[1] + FB[1])) * irt;
                u_out[(size_t)2 * p.N + n] = (jz + 0.5f * (FA[2] + FB[2])) * irt;
            }
        }
#pragma unroll
        for (int i = 0; i < 2 * Q; i++) cur[i] = nxt[i];
    }
}

constexpr int BTX = 32, BTY = 8;

static void bulk_geometry(const LbmParams& p, dim3& grid, int& threads) {
    int nzf = p.zf1 - p.zf0;
    grid = dim3((p.nx + BTX - 1) / BTX, (p.ny + BTY - 1) / BTY, (nzf + p.lz - 1) / p.lz);
    threads = Tile<BTX, BTY>::HN;
}

int bulk_grid_blocks(const LbmParams& p) {
    dim3 g;
    int th;
    bulk_geometry(p, g, th);
    return (int)(g.x * g.y * g.z);
}

void launch_bulk(const LbmParams& p, const float* S, float* D, float* rho, const float* ghost, const float* Fibm,
                 const uint32_t* mask, float* u, int* err, bool ibm, cudaStream_t st) {
    dim3 grid;
    int threads;
    bulk_geometry(p, grid, threads);
    if (ibm)
        k_bulk<BTX, BTY, true><<<grid, threads, 0, st>>>(p, S, D, rho, ghost, Fibm, mask, u, err);
    else
        k_bulk<BTX, BTY, false><<<grid, threads, 0, st>>>(p, S, D, rho, ghost, Fibm, mask, u, err);
}

void launch_init_state(const LbmParams& p, float* S, const float* rho_st, const float* u_st, cudaStream_t st) {
    k_init_state<<<(p.N + 255) / 256, 256, 0, st>>>(p, S, rho_st, u_st);
}

void launch_wall_ghost(const LbmParams& p, const float* S, float* wall_rho, float* ghost, cudaStream_t st) {
    k_wall_planes_rho<<<(2 * p.nxy + 255) / 256, 256, 0, st>>>(p, S, wall_rho);
    k_wall_ghost<<<(4 * p.nxy + 255) / 256, 256, 0, st>>>(p, wall_rho, ghost);
}

// ------------------------------------------------------------------------------------------------------
// Exports of the current state.  what = 0: rho^A, rho^B, u (5 N floats); what = 1: populations in the
// [c][node][i] order (38 N floats).  Wall nodes report 0.
// ------------------------------------------------------------------------------------------------------
__global__ void k_export(LbmParams p, const float* __restrict__ S, float* __restrict__ out, int what) {
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
    }
    if (what == 1) {
#pragma unroll
        for (int i = 0; i < Q; i++) {
            out[(size_t)n * Q + i] = f[i];
            out[(size_t)(p.N + n) * Q + i] = f[Q + i];
        }
        return;
    }
    float ra = 0.f, rb = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        ra += f[i]; rb += f[Q + i];
        const float fs = f[i] + f[Q + i];
        jx += dir_x(i) * fs; jy += dir_y(i) * fs; jz += dir_z(i) * fs;
    }
    const float rt = ra + rb;
    const float irt = rt > 0.f ? 1.f / rt : 0.f;
    out[n] = ra;
    out[p.N + n] = rb;
    out[2 * (size_t)p.N + n] = jx * irt;
    out[3 * (size_t)p.N + n] = jy * irt;
    out[4 * (size_t)p.N + n] = jz * irt;
}

void launch_export(const LbmParams& p, const float* S, float* out, int what, cudaStream_t st) {
    k_export<<<(p.N + 255) / 256, 256, 0, st>>>(p, S, out, what);
}

// ------------------------------------------------------------------------------------------------------
// FP64 reductions of the current state: mass per component and total momentum (fixed order: per-block
// partials, then one block sums them), red[0..4] = M^A, M^B, P_x, P_y, P_z.
// ------------------------------------------------------------------------------------------------------
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 1024;

__global__ void __launch_bounds__(RED_THREADS) k_moments_partial(LbmParams p, const float* __restrict__ S,
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
    k_moments_partial<<<RED_BLOCKS, RED_THREADS, 0, st>>>(p, S, red + 8);
    k_sum_partials<<<1, RED_THREADS, 0, st>>>(red + 8, RED_BLOCKS, 5, red);
}

}  // namespace scbb
