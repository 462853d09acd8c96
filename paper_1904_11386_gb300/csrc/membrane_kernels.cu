// Membrane kernels of libscbb (sm_103a): Skalak strain (Eq. 6, 8), volume penalty (Eq. 7), Helfrich bending
// with the discrete operators of Meyer et al. (Eq. 9-10), FP64 capsule reductions, 2-point immersed-boundary
// spreading / interpolation, and the particle-particle repulsion (Eq. 26).
//
// Forces are gathered per vertex over its incident triangles (a vertex -> triangle CSR), so every vertex
// sums its contributions in a fixed order: no atomics, bitwise reproducible.  A triangle's terms are
// recomputed by each of its three vertices, which costs nothing measurable at these mesh sizes.
#include <math.h>

#include "membrane.cuh"
#include "pdl.cuh"
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
// sum unchanged but keeps the FP32 triple products small) and centre of mass.  The per-triangle terms are
// FP32, the sums FP64 (GB300's FP64 rate is low, so only the accumulation is double).  Fixed order.
// ------------------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

constexpr int CAP_THREADS = 1024;

// Volume terms come from the triangle pass (tvol), so the reduction is a plain FP64 sum.
__global__ void __launch_bounds__(CAP_THREADS) k_capsule_reduce(DevState d, int use_tvol) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh[4 * 32];
    const int m = blockIdx.x;
    const CapDev c = d.cap[m];
    // per-thread and per-warp partials in FP32 (a few dozen terms each), the block sum in FP64
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (use_tvol) {
#pragma unroll 4
        for (int t = threadIdx.x; t < c.nt; t += blockDim.x) acc[0] += d.tvol[c.t0 + t];
    } else {
        const float3 r0 = ld3(d.X[c.v0]);
        for (int t = threadIdx.x; t < c.nt; t += blockDim.x) {
            const int4 T = d.tri[c.t0 + t];
            const float3 a = ld3(d.X[T.x]) - r0, b = ld3(d.X[T.y]) - r0, e = ld3(d.X[T.z]) - r0;
            acc[0] += dotf(a, crossf(b, e)) * (1.f / 6.f);
        }
    }
    float mn[3] = {1e30f, 1e30f, 1e30f}, mx[3] = {-1e30f, -1e30f, -1e30f};
    const float4 r0c = d.X[c.v0];       // vertex sums relative to the first vertex (small FP32 terms)
#pragma unroll 4
    for (int v = threadIdx.x; v < c.nv; v += blockDim.x) {
        const float4 q = d.X[c.v0 + v];
        acc[1] += q.x - r0c.x; acc[2] += q.y - r0c.y; acc[3] += q.z - r0c.z;
        mn[0] = fminf(mn[0], q.x); mn[1] = fminf(mn[1], q.y); mn[2] = fminf(mn[2], q.z);
        mx[0] = fmaxf(mx[0], q.x); mx[1] = fmaxf(mx[1], q.y); mx[2] = fmaxf(mx[2], q.z);
    }
    __shared__ float shb[6 * 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float s = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[k * 32 + w] = (double)s;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float a = mn[k], b = mx[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fminf(a, __shfl_down_sync(0xffffffffu, a, o));
            b = fmaxf(b, __shfl_down_sync(0xffffffffu, b, o));
        }
        if (lane == 0) { shb[k * 32 + w] = a; shb[(3 + k) * 32 + w] = b; }
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const double s = warp_sum(lane < nw ? sh[k * 32 + lane] : 0.0);
            const double r0k = k == 1 ? r0c.x : (k == 2 ? r0c.y : r0c.z);
            if (lane == 0) d.cap_red[4 * m + k] = k == 0 ? s : s / c.nv + r0k;
        }
        if (d.cbox) {
            // classification box: vertex bounds padded by 3 nodes (covers the next step's positions)
            int lo[3], hi[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                float a = lane < nw ? shb[k * 32 + lane] : 1e30f, b = lane < nw ? shb[(3 + k) * 32 + lane] : -1e30f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a = fminf(a, __shfl_down_sync(0xffffffffu, a, o));
                    b = fmaxf(b, __shfl_down_sync(0xffffffffu, b, o));
                }
                a = fmaxf(a, -1e6f);
                b = fminf(b, 1e6f);
                lo[k] = (int)floorf(a) - 3;
                hi[k] = (int)ceilf(b) + 3;
            }
            if (lane == 0) {
                bool over = false;
                for (int k = 0; k < 3; k++)
                    if (hi[k] - lo[k] + 1 > d.CW) { hi[k] = lo[k] + d.CW - 1; over = true; }
                if (over) atomicOr(d.cnt + 2, 16);
                d.cbox[2 * m] = make_int4(lo[0], lo[1], lo[2], 0);
                d.cbox[2 * m + 1] = make_int4(hi[0], hi[1], hi[2], 0);
            }
        }
    }
}

void launch_capsule_reduce(const DevState& d, cudaStream_t st) {
    if (d.NM > 0) launch_k(k_capsule_reduce, dim3(d.NM), dim3(CAP_THREADS), 0, st, d, 0);
}

// ------------------------------------------------------------------------------------------------------
// Membrane forces in three grid-parallel passes plus the FP64 capsule reduction:
//   triangle pass  Skalak force on each corner (Eq. 6; F = -dE/dx of Eq. 8 through the metric invariants
//                  tr(g0^-1 g) and det g / det g0), volume gradient (x_j - r0) x (x_l - r0)/6 and volume
//                  term, Meyer terms: angle, cotangents of the two other angles, mixed-area share, the
//                  corner's share of the mean-curvature normal, face normal
//   vertex pass 1  gather the corners of a vertex -> mixed area A, unit normal n, H = (K . n)/2 with
//                  K = (1/2A) sum (cot a + cot b)(x_i - x_j), Gaussian curvature (2 pi - sum of angles)/A
//   reduction      capsule volume and centre of mass (FP64)
//   vertex pass 2  Laplace-Beltrami of H, bending force 2 kB [2H(H^2 - K) + Lap H] A n (Eq. 10), volume
//                  force -kV (V - V0)/V0 dV/dx (Eq. 7-8), total elastic force
// The vertex passes gather through a vertex -> corner CSR in a fixed order (no atomics, reproducible) and
// prefetch a vertex's corner ids before the records, so each gather costs two or three dependent loads.
// Corner c = 3 t + k of triangle t; cnb[c] holds the global ids of the two other corners (j, l).
// ------------------------------------------------------------------------------------------------------
__global__ void k_mem_tri(DevState d) {
    pdl_wait();
    pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d.NT) return;
    const int4 T = d.tri[t];
    const CapDev cp = d.cap[T.w];
    const float3 r0 = ld3(d.X[cp.v0]);
    const float4 R = d.tref[t];                       // (ia, ib, ic, A0): inverse reference metric, area
    const float3 P[3] = {ld3(d.X[T.x]), ld3(d.X[T.y]), ld3(d.X[T.z])};
    const float3 e1 = P[1] - P[0], e2 = P[2] - P[0];
    const float g11 = dotf(e1, e1), g12 = dotf(e1, e2), g22 = dotf(e2, e2);
    const float idet0 = R.x * R.z - R.y * R.y;        // 1 / det(g0)
    const float I1 = R.x * g11 + 2.f * R.y * g12 + R.z * g22 - 2.f;
    const float I2 = (g11 * g22 - g12 * g12) * idet0 - 1.f;
    const float pre = 0.25f * cp.kS * R.w;
    const float d1 = pre * (2.f * I1 + 2.f), d2 = pre * (2.f * cp.C * I2 - 2.f);
    const float W11 = d1 * R.x + d2 * g22 * idet0;
    const float W12 = 2.f * d1 * R.y - 2.f * d2 * g12 * idet0;
    const float W22 = d1 * R.z + d2 * g11 * idet0;
    const float3 G1 = (2.f * W11) * e1 + W12 * e2;       // dE/de1
    const float3 G2 = W12 * e1 + (2.f * W22) * e2;       // dE/de2
    const float3 Fc[3] = {G1 + G2, -1.f * G1, -1.f * G2};
    const float3 nrm = crossf(e1, e2);                   // 2 * area * outward unit normal
    const float s2 = sqrtf(dotf(nrm, nrm));
    const float area = 0.5f * s2;
    float dots[3], cots[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float3 a = P[(k + 1) % 3] - P[k], b = P[(k + 2) % 3] - P[k];
        dots[k] = dotf(a, b);
        cots[k] = dots[k] / s2;
    }
    const int obtuse = dots[0] < 0.f ? 0 : (dots[1] < 0.f ? 1 : (dots[2] < 0.f ? 2 : -1));
    const float3 pa = P[0] - r0, pb = P[1] - r0, pc = P[2] - r0;
    d.tvol[t] = dotf(pa, crossf(pb, pc)) * (1.f / 6.f);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int j = (k + 1) % 3, l = (k + 2) % 3;
        const float3 aij = P[j] - P[k], ail = P[l] - P[k];
        // edge (i, j) is opposite corner l, edge (i, l) opposite corner j
        const float3 K = (-cots[l]) * aij + (-cots[j]) * ail;
        float Ash;
        if (obtuse < 0) Ash = 0.125f * (cots[l] * dotf(aij, aij) + cots[j] * dotf(ail, ail));
        else Ash = (obtuse == k) ? 0.5f * area : 0.25f * area;
        const float th = atan2f(s2, dots[k]);
        const float3 dv = (1.f / 6.f) * crossf(P[j] - r0, P[l] - r0);
        float4* rec = d.corner + 4 * (3 * t + k);
        rec[0] = make_float4(Fc[k].x, Fc[k].y, Fc[k].z, Ash);
        rec[1] = make_float4(dv.x, dv.y, dv.z, th);
        rec[2] = make_float4(K.x, K.y, K.z, 0.f);
        rec[3] = make_float4(nrm.x, nrm.y, nrm.z, 0.f);
        d.ccot[3 * t + k] = make_float2(cots[j], cots[l]);
    }
}

constexpr int GATHER = 8;      // corners fetched per round of a vertex gather

__global__ void k_mem_vert1(DevState d) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.NV) return;
    float3 Fs = make_float3(0.f, 0.f, 0.f), dv = make_float3(0.f, 0.f, 0.f), K = make_float3(0.f, 0.f, 0.f);
    float3 nn = make_float3(0.f, 0.f, 0.f);
    float A = 0.f, ang = 0.f;
    const int q0 = d.vt_off[i], q1 = d.vt_off[i + 1];
    for (int qb = q0; qb < q1; qb += GATHER) {
        int cid[GATHER];
#pragma unroll
        for (int u = 0; u < GATHER; u++) cid[u] = qb + u < q1 ? d.vt_idx[qb + u] : -1;
#pragma unroll
        for (int u = 0; u < GATHER; u++) {
            if (cid[u] < 0) continue;
            const float4* rec = d.corner + 4 * cid[u];
            const float4 a = rec[0], b = rec[1], c = rec[2], e = rec[3];
            Fs = Fs + make_float3(a.x, a.y, a.z);
            A += a.w;
            dv = dv + make_float3(b.x, b.y, b.z);
            ang += b.w;
            K = K + make_float3(c.x, c.y, c.z);
            nn = nn + make_float3(e.x, e.y, e.z);
        }
    }
    nn = rsqrtf(dotf(nn, nn)) * nn;
    K = (0.5f / A) * K;
    const float H = 0.5f * dotf(K, nn);
    const float KG = (6.283185307179586f - ang) / A;
    d.Fsk[i] = make_float4(Fs.x, Fs.y, Fs.z, 0.f);
    d.dV[i] = make_float4(dv.x, dv.y, dv.z, 0.f);
    d.nrm[i] = make_float4(nn.x, nn.y, nn.z, H);
    d.AK[i] = make_float2(A, KG);
}

// bb: add the bounce-back coupling (exchanged momentum smoothed over two steps, Shan-Chen reactions and
// fresh-node momenta of the crossed elements, one third to each corner) and advance the node
// (V += F/m, then X += V).
__global__ void k_mem_vert2(DevState d, int bb, int step) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.NV) return;
    const int m = d.vcap[i];
    const CapDev cp = d.cap[m];
    const float4 ni = d.nrm[i];
    const float Hi = ni.w;
    float lap = 0.f;
    float cx = 0.f, cy = 0.f, cz = 0.f;                // bounce-back coupling of the adjacent elements
    const int now = step & 1, prev = (step + 1) & 1;
    const int q0 = d.vt_off[i], q1 = d.vt_off[i + 1];
    for (int qb = q0; qb < q1; qb += GATHER) {
        int cid[GATHER];
#pragma unroll
        for (int u = 0; u < GATHER; u++) cid[u] = qb + u < q1 ? d.vt_idx[qb + u] : -1;
#pragma unroll
        for (int u = 0; u < GATHER; u++) {
            if (cid[u] < 0) continue;
            const int2 nb = d.cnb[cid[u]];
            const float2 ct = d.ccot[cid[u]];          // (cot at j, cot at l)
            // edge (i, j) carries the cotangent of the angle at l, edge (i, l) that at j
            lap += ct.y * (d.nrm[nb.x].w - Hi) + ct.x * (d.nrm[nb.y].w - Hi);
            if (bb) {
                const int e = cid[u] / 3;
                const float4 a = d.emom[now * d.NT + e], b = d.emom[prev * d.NT + e], c = d.epend[now * d.NT + e];
                cx += 0.5f * (a.x + b.x) + c.x;
                cy += 0.5f * (a.y + b.y) + c.y;
                cz += 0.5f * (a.z + b.z) + c.z;
            }
        }
    }
    const float2 AK = d.AK[i];
    lap *= 0.5f / AK.x;
    const float fb = 2.f * cp.kB * (2.f * Hi * (Hi * Hi - AK.y) + lap) * AK.x;
    const float kv = (float)(-(double)cp.kV * (d.cap_red[4 * m] - cp.V0) / cp.V0);
    const float4 fs = d.Fsk[i], dvv = d.dV[i];
    float4 F = make_float4(fs.x + fb * ni.x + kv * dvv.x, fs.y + fb * ni.y + kv * dvv.y,
                           fs.z + fb * ni.z + kv * dvv.z, 0.f);
    if (d.pp_head) {                                   // particle-particle repulsion (Eq. 26)
        const float4 fp = d.Fpp[i];
        F.x += fp.x; F.y += fp.y; F.z += fp.z;
    }
    if (bb) {
        F.x += cx * (1.f / 3.f); F.y += cy * (1.f / 3.f); F.z += cz * (1.f / 3.f);
        float4 V = d.V[i], X = d.X[i];
        const float im = 1.f / cp.mass;
        V.x += F.x * im; V.y += F.y * im; V.z += F.z * im;
        X.x += V.x; X.y += V.y; X.z += V.z;
        d.V[i] = V;
        d.X[i] = X;
    }
    d.F[i] = F;
}

int launch_membrane_elastic(const LbmParams& p, const DevState& d, cudaStream_t st) {
    if (d.NM == 0) return 0;
    const int b = 128;
    const int npp = launch_pp_forces(p, d, d.pp_eps, d.pp_d0, st);
    launch_k(k_mem_tri, dim3((d.NT + b - 1) / b), dim3(b), 0, st, d);
    launch_k(k_mem_vert1, dim3((d.NV + b - 1) / b), dim3(b), 0, st, d);
    launch_k(k_capsule_reduce, dim3(d.NM), dim3(CAP_THREADS), 0, st, d, 1);
    return 3 + npp;
}

int launch_membrane_update(const LbmParams& p, const DevState& d, bool bb, int step, cudaStream_t st) {
    if (d.NM == 0) return 0;
    const int b = 128;
    launch_k(k_mem_vert2, dim3((d.NV + b - 1) / b), dim3(b), 0, st, d, bb ? 1 : 0, step);
    return 1;
}

int launch_membrane_forces(const LbmParams& p, const DevState& d, bool bb, int step, cudaStream_t st) {
    return launch_membrane_elastic(p, d, st) + launch_membrane_update(p, d, bb, step, st);
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
    if ((unsigned)a < (unsigned)n) return a;        // in range: no integer modulo
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

// Spreading (Eq. 9 forces onto the lattice): the vertices' contributions w F are summed into the fixed-point
// force field (ibm_fix: integer atomics, so the sums do not depend on the order the atomics land in), and the
// nodes they reach are marked.
__global__ void k_ibm_spread(LbmParams p, DevState d) {
    pdl_wait();
    pdl_trigger();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= d.NV) return;
    const Stencil s = hat_stencil(p, d.X[v]);
    const float4 F = d.F[v];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if (!s.fluid[q]) continue;
        const unsigned int n = s.node[q];
        atomicAdd(d.Fibm + n, ibm_fix(s.w[q] * F.x));
        atomicAdd(d.Fibm + (size_t)p.N + n, ibm_fix(s.w[q] * F.y));
        atomicAdd(d.Fibm + 2 * (size_t)p.N + n, ibm_fix(s.w[q] * F.z));
        atomicOr(d.mask + (n >> 5), 1u << (n & 31));
    }
}

// Reads the velocity at the stencil of the current position, clears the force field and the marks of that
// stencil (nothing else reads them in this kernel), then moves the vertex.  Wall nodes contribute the wall
// velocity.
__global__ void k_ibm_interp(LbmParams p, DevState d) {
    pdl_wait();
    pdl_trigger();
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
            for (int k = 0; k < 3; k++) d.Fibm[(size_t)k * p.N + n] = 0ull;
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

int launch_ibm_spread(const LbmParams& p, const DevState& d, cudaStream_t st) {
    if (d.NV == 0) return 0;
    launch_k(k_ibm_spread, dim3((d.NV + 127) / 128), dim3(128), 0, st, p, d);
    return 1;
}

void launch_ibm_interp(const LbmParams& p, const DevState& d, cudaStream_t st) {
    if (d.NV == 0) return;
    launch_k(k_ibm_interp, dim3((d.NV + 127) / 128), dim3(128), 0, st, p, d);
}

// ------------------------------------------------------------------------------------------------------
// Particle-particle repulsion (Eq. 26): nodes of different capsules closer than d0 push each other apart
// with eps (d0 - d)^{3/2} along their separation (minimum image in the periodic directions).  Vertices go
// into a hashed grid of cells at least d0 wide (linked lists, head table of 2^k >= 2 NV entries); every
// vertex then gathers over the 27 cells around it.  Hash collisions only add candidates that the distance
// test rejects.  The gather sums each vertex's own force, so Newton's third law holds pairwise.
// ------------------------------------------------------------------------------------------------------
struct PPGrid {
    int nc[3];          // cells per direction (periodic directions wrap)
    float cw[3];        // cell widths (>= d0)
    int per[3];
    float L[3];
    unsigned mask;      // hash table size - 1
};

__device__ __forceinline__ unsigned pp_hash(int cx, int cy, int cz, unsigned mask) {
    return ((unsigned)cx * 73856093u ^ (unsigned)cy * 19349663u ^ (unsigned)cz * 83492791u) & mask;
}

__device__ __forceinline__ int pp_cell(float v, int k, const PPGrid& g) {
    if (g.per[k]) {
        v = fmodf(v, g.L[k]);
        if (v < 0.f) v += g.L[k];
    }
    int c = (int)floorf(v / g.cw[k]);
    if (g.per[k]) c = c < 0 ? 0 : (c >= g.nc[k] ? g.nc[k] - 1 : c);
    return c;
}

// Empty hash table; each capsule's reference point for this step (its centre, as the last reduction left it)
// and a zero bounding radius.
__global__ void k_pp_clear(DevState d, unsigned size) {
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < size; q += gridDim.x * blockDim.x) d.pp_head[q] = -1;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d.NM; k += gridDim.x * blockDim.x) {
        const double* cr = d.cap_red + 4 * k;
        d.pp_ref[k] = make_float4((float)cr[1], (float)cr[2], (float)cr[3], 0.f);
        d.pp_rmax[k] = 0;
    }
}

// minimum-image separation a - b
__device__ __forceinline__ float3 pp_sep(float3 a, float3 b, const PPGrid& g) {
    float r[3] = {a.x - b.x, a.y - b.y, a.z - b.z};
    for (int k = 0; k < 3; k++)
        if (g.per[k]) r[k] -= g.L[k] * floorf(r[k] / g.L[k] + 0.5f);
    return make_float3(r[0], r[1], r[2]);
}

// Margin of the sphere tests over the rounding of these FP32 distances.
constexpr float PP_MARGIN = 1e-3f;

// Per capsule: the other capsules whose bounding spheres (reference point, largest vertex distance) come within
// the repulsion range d0 of its own.  A vertex farther than radius + d0 from every such capsule's reference
// point has no vertex of another capsule within d0 (triangle inequality of the minimum-image distance).
// One warp per capsule i, its lanes over the other capsules j.
__global__ void k_pp_pairs(DevState d, PPGrid g, float d0) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= d.NM) return;                          // warp-uniform
    const float4 ci = d.pp_ref[i];
    const float ri = __int_as_float(d.pp_rmax[i]);
    int n = 0;
    for (int j0 = 0; j0 < d.NM; j0 += 32) {
        const int j = j0 + lane;
        bool hit = false;
        if (j < d.NM && j != i) {
            const float4 cj = d.pp_ref[j];
            const float3 r = pp_sep(make_float3(ci.x, ci.y, ci.z), make_float3(cj.x, cj.y, cj.z), g);
            const float reach = ri + __int_as_float(d.pp_rmax[j]) + d0 + PP_MARGIN;
            hit = !(r.x * r.x + r.y * r.y + r.z * r.z > reach * reach);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        const int at = n + __popc(bal & ((1u << lane) - 1u));
        if (hit && at < PP_NBR) d.pp_nbr[i * PP_NBR + at] = j;
        n += __popc(bal);
    }
    // too many: the vertices of capsule i search without the filter
    if (lane == 0) d.pp_ncnt[i] = n > PP_NBR ? -1 : n;
}

__global__ void k_pp_insert(DevState d, PPGrid g) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int k = -1;
    float dist = 0.f;
    if (v < d.NV) {
        const float4 X = d.X[v];
        if (!(fabsf(X.x) < 1e6f && fabsf(X.y) < 1e6f && fabsf(X.z) < 1e6f)) {
            d.pp_next[v] = -1;
        } else {
            const unsigned h = pp_hash(pp_cell(X.x, 0, g), pp_cell(X.y, 1, g), pp_cell(X.z, 2, g), g.mask);
            d.pp_next[v] = atomicExch(d.pp_head + h, v);
            k = d.vcap[v];
            const float4 c = d.pp_ref[k];
            const float3 r = pp_sep(make_float3(X.x, X.y, X.z), make_float3(c.x, c.y, c.z), g);
            dist = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
        }
    }
    // the capsule's bounding radius: one atomic per warp when the warp's vertices share a capsule (they are
    // stored capsule by capsule), else one per vertex; distances are >= 0, so their bits order as ints
    const int k0 = __shfl_sync(0xffffffffu, k, 0);
    if (__all_sync(0xffffffffu, k == k0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dist = fmaxf(dist, __shfl_xor_sync(0xffffffffu, dist, o));
        if (lane == 0 && k0 >= 0) atomicMax(d.pp_rmax + k0, __float_as_int(dist));
    } else if (k >= 0) {
        atomicMax(d.pp_rmax + k, __float_as_int(dist));
    }
}

__global__ void k_pp_force(DevState d, PPGrid g, float eps, float d0) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= d.NV) return;
    const float4 X = d.X[v];
    const int cap = d.vcap[v];
    float3 F = make_float3(0.f, 0.f, 0.f);
    // the cell search only where another capsule's bounding sphere comes within d0 (else no term is nonzero)
    const int nn = d.pp_ncnt[cap];
    bool near = nn < 0;
    for (int q = 0; q < nn && !near; q++) {
        const int j = d.pp_nbr[cap * PP_NBR + q];
        const float4 c = d.pp_ref[j];
        const float3 r = pp_sep(make_float3(X.x, X.y, X.z), make_float3(c.x, c.y, c.z), g);
        const float reach = __int_as_float(d.pp_rmax[j]) + d0 + PP_MARGIN;
        near = !(r.x * r.x + r.y * r.y + r.z * r.z > reach * reach);     // a non-finite distance searches
    }
    if (near && fabsf(X.x) < 1e6f && fabsf(X.y) < 1e6f && fabsf(X.z) < 1e6f) {
        const int c0[3] = {pp_cell(X.x, 0, g), pp_cell(X.y, 1, g), pp_cell(X.z, 2, g)};
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int cc[3] = {c0[0] + dx, c0[1] + dy, c0[2] + dz};
                    const int dd[3] = {dx, dy, dz};
                    bool skip = false;
                    for (int k = 0; k < 3; k++) {
                        if (g.per[k]) {
                            if (g.nc[k] < 3 && dd[k] != 0 && (g.nc[k] == 1 || dd[k] == 1)) skip = true;  // no revisit
                            cc[k] = cc[k] < 0 ? cc[k] + g.nc[k] : (cc[k] >= g.nc[k] ? cc[k] - g.nc[k] : cc[k]);
                        }
                    }
                    if (skip) continue;
                    const unsigned h = pp_hash(cc[0], cc[1], cc[2], g.mask);
                    for (int w = d.pp_head[h]; w >= 0; w = d.pp_next[w]) {
                        if (d.vcap[w] == cap) continue;
                        const float4 Y = d.X[w];
                        float r[3] = {X.x - Y.x, X.y - Y.y, X.z - Y.z};
                        for (int k = 0; k < 3; k++)
                            if (g.per[k]) r[k] -= g.L[k] * floorf(r[k] / g.L[k] + 0.5f);
                        // only the cell this neighbour really occupies counts (hash collisions)
                        const int wc[3] = {pp_cell(Y.x, 0, g), pp_cell(Y.y, 1, g), pp_cell(Y.z, 2, g)};
                        if (wc[0] != cc[0] || wc[1] != cc[1] || wc[2] != cc[2]) continue;
                        const float dist = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                        if (dist < d0 && dist > 0.f) {
                            const float q = d0 - dist;
                            const float mag = eps * q * sqrtf(q) / dist;
                            F.x += mag * r[0]; F.y += mag * r[1]; F.z += mag * r[2];
                        }
                    }
                }
    }
    d.Fpp[v] = make_float4(F.x, F.y, F.z, 0.f);
}

int launch_pp_forces(const LbmParams& p, const DevState& d, float eps, float d0, cudaStream_t st) {
    if (!d.pp_head || d.NM < 2 || eps == 0.f) return 0;
    PPGrid g;
    const float L[3] = {(float)p.nx, (float)p.ny, (float)p.nz};
    const int per[3] = {1, 1, p.walls ? 0 : 1};
    for (int k = 0; k < 3; k++) {
        g.per[k] = per[k];
        g.L[k] = L[k];
        int n = (int)floorf(L[k] / d0);
        if (n < 1) n = 1;
        g.nc[k] = n;
        g.cw[k] = per[k] ? L[k] / n : d0;       // non-periodic z: unbounded cells of width d0
    }
    g.mask = (unsigned)d.pp_size - 1u;
    k_pp_clear<<<(d.pp_size + 255) / 256, 256, 0, st>>>(d, (unsigned)d.pp_size);
    k_pp_insert<<<(d.NV + 127) / 128, 128, 0, st>>>(d, g);
    k_pp_pairs<<<(d.NM * 32 + 127) / 128, 128, 0, st>>>(d, g, d0);
    k_pp_force<<<(d.NV + 127) / 128, 128, 0, st>>>(d, g, eps, d0);
    return 4;
}

}  // namespace scbb
