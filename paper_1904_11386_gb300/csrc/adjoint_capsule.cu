// Adjoint of a capsule coupled to the fluid by the 2-point immersed boundary (sm_103a): the parts of one step
// backwards that the fluid adjoint (adjoint_kernels.cu) does not cover.
//
// Forward step t (the context's immersed-boundary step): node forces F(X) of the membrane (Skalak Eq. 6-8, volume
// Eq. 7, Helfrich-Meyer bending Eq. 9-10), spread onto the lattice Fibm(x) = sum_b phi(x - X_b) F_b, the fluid step
// with that force (its half-force velocity uh written at the marked nodes), then X_b += sum_x phi(x - X_b) uh(x)
// (wall nodes of the stencil contribute the wall velocity).  With lambda_X the adjoint of X(t + 1):
//   spread      luh(x) = sum_b phi(x - X_b) lambda_X,b          (the interpolation transposed)
//   fluid       local and push passes with luh in, lambda_Fibm out (adjoint_kernels.cu)
//   vertex      lambda_F,b = sum_x phi(x - X_b) lambda_Fibm(x)    (the spreading transposed)
//               lambda_X,b += sum_x grad phi(x - X_b) [uh(x) . lambda_X,b + lambda_Fibm(x) . F_b]
//   membrane    lambda_X += (dF/dX)^T lambda_F: per triangle, the corner forces and records of the forward triangle
//               pass evaluated with 9-direction dual numbers (the triangle's coordinates), contracted with their
//               adjoints; bending's vertex stages (mixed area, normal, H, Gaussian curvature, Laplace-Beltrami of
//               H) reversed by hand in two vertex passes before it
//   parameters  dL/dkS += lambda_F . F_Skalak / kS (the force is linear in kS), likewise kB and kV.
// All arithmetic FP32; the parameter sums FP64.
#include <math.h>

#include "adjoint.cuh"
#include "scbb_internal.cuh"
#include "pdl.cuh"

namespace scbb {

namespace {

// ---- 9-direction dual numbers
struct D9 {
    float v;
    float d[9];
};
__device__ __forceinline__ D9 dc(float v) {
    D9 r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < 9; k++) r.d[k] = 0.f;
    return r;
}
__device__ __forceinline__ D9 operator+(const D9& a, const D9& b) {
    D9 r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < 9; k++) r.d[k] = a.d[k] + b.d[k];
    return r;
}
__device__ __forceinline__ D9 operator-(const D9& a, const D9& b) {
    D9 r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < 9; k++) r.d[k] = a.d[k] - b.d[k];
    return r;
}
__device__ __forceinline__ D9 operator*(const D9& a, const D9& b) {
    D9 r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < 9; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
__device__ __forceinline__ D9 operator*(float s, const D9& a) {
    D9 r;
    r.v = s * a.v;
#pragma unroll
    for (int k = 0; k < 9; k++) r.d[k] = s * a.d[k];
    return r;
}
__device__ __forceinline__ D9 operator+(const D9& a, float s) {
    D9 r = a;
    r.v += s;
    return r;
}
__device__ __forceinline__ D9 operator/(const D9& a, const D9& b) {
    const float ib = 1.f / b.v;
    D9 r;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < 9; k++) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
__device__ __forceinline__ D9 dsqrt(const D9& a) {
    D9 r;
    r.v = sqrtf(a.v);
    const float h = 0.5f / r.v;
#pragma unroll
    for (int k = 0; k < 9; k++) r.d[k] = h * a.d[k];
    return r;
}
__device__ __forceinline__ D9 datan2(const D9& y, const D9& x) {   // d atan2(y, x) = (x dy - y dx) / (x^2 + y^2)
    D9 r;
    r.v = atan2f(y.v, x.v);
    const float q = 1.f / (x.v * x.v + y.v * y.v);
#pragma unroll
    for (int k = 0; k < 9; k++) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * q;
    return r;
}
struct V9 {
    D9 x, y, z;
};
__device__ __forceinline__ V9 operator-(const V9& a, const V9& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V9 operator+(const V9& a, const V9& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V9 operator*(const D9& s, const V9& a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ V9 operator*(float s, const V9& a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ D9 vdot(const V9& a, const V9& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V9 vcross(const V9& a, const V9& b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// contraction lambda . dv/dP[k] of a dual vector with a float adjoint
__device__ __forceinline__ float vcon(const float4 l, const V9& a, int k) {
    return l.x * a.x.d[k] + l.y * a.y.d[k] + l.z * a.z.d[k];
}

// ---- hat stencil of the immersed boundary with the gradient of each weight with respect to the vertex
struct AdjStencil {
    unsigned int node[8];
    float w[8];
    float gw[8][3];
    bool fluid[8];
    bool wall[8];
    int zc[8];
};
__device__ __forceinline__ int wrapn(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    a %= n;
    return a < 0 ? a + n : a;
}
__device__ __forceinline__ AdjStencil adj_stencil(const LbmParams& p, float4 X) {
    AdjStencil s;
    const float fx = floorf(X.x), fy = floorf(X.y), fz = floorf(X.z);
    const float rx = X.x - fx, ry = X.y - fy, rz = X.z - fz;
    const int bx = (int)fx, by = (int)fy, bz = (int)fz;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int dx = q & 1, dy = (q >> 1) & 1, dz = q >> 2;
        const int xx = wrapn(bx + dx, p.nx), yy = wrapn(by + dy, p.ny);
        int zz = bz + dz;
        if (!p.walls) zz = wrapn(zz, p.nz);
        const bool inside = zz >= 0 && zz < p.nz;
        const bool wall = inside && p.walls && (zz == 0 || zz == p.nz - 1);
        s.zc[q] = zz;
        s.fluid[q] = inside && !wall;
        s.wall[q] = wall;
        s.node[q] = inside ? (unsigned int)(xx + p.nx * (yy + p.ny * zz)) : 0u;
        const float wx = dx ? rx : 1.f - rx, wy = dy ? ry : 1.f - ry, wz = dz ? rz : 1.f - rz;
        const float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
        s.w[q] = inside ? wx * wy * wz : 0.f;
        s.gw[q][0] = inside ? sx * wy * wz : 0.f;
        s.gw[q][1] = inside ? wx * sy * wz : 0.f;
        s.gw[q][2] = inside ? wx * wy * sz : 0.f;
    }
    return s;
}

// volume factor kv = -kV (V - V0) / V0 of a capsule (Eq. 7)
__device__ __forceinline__ float volume_factor(const DevState& d, int m) {
    const CapDev c = d.cap[m];
    return (float)(-(double)c.kV * (d.cap_red[4 * m] - c.V0) / c.V0);
}

}  // namespace

// luh(x) += phi(x - X_b) lambda_X,b over the fluid nodes of each vertex's stencil (the interpolation transposed)
__global__ void k_cap_adj_spread(LbmParams p, DevState d, AdjCap a) {
    pdl_wait();
    pdl_trigger();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < d.NM) a.capd[4 * v + 3] = 0.0;             // the step's lambda_F . dV, summed by k_cap_adj_vert
    if (v >= d.NV) return;
    const AdjStencil s = adj_stencil(p, d.X[v]);
    const float4 l = a.lx[v];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if (!s.fluid[q]) continue;
        const unsigned int n = s.node[q];
        atomicAdd(a.luh + n, s.w[q] * l.x);
        atomicAdd(a.luh + (size_t)p.N + n, s.w[q] * l.y);
        atomicAdd(a.luh + 2 * (size_t)p.N + n, s.w[q] * l.z);
    }
}

// Per vertex: the adjoint of its node force (the spreading transposed), the stencil terms of lambda_X, and the
// first reverse stage of bending; the per-vertex products that the capsule reduction sums.
__global__ void k_cap_adj_vert(LbmParams p, DevState d, AdjCap a) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.NV) return;
    const float4 X = d.X[i];
    const AdjStencil s = adj_stencil(p, X);
    const float4 lX = a.lx[i];
    const float4 F = d.F[i];
    float lF[3] = {0.f, 0.f, 0.f}, g[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const unsigned int n = s.node[q];
        float u[3] = {0.f, 0.f, 0.f}, lf[3] = {0.f, 0.f, 0.f};
        if (s.fluid[q]) {
            for (int k = 0; k < 3; k++) {
                u[k] = a.uh[(size_t)k * p.N + n];
                lf[k] = a.lfi[(size_t)k * p.N + n];
            }
        } else if (s.wall[q]) {
            const float* Uw = s.zc[q] == 0 ? p.ulo : p.uhi;
            u[0] = Uw[0]; u[1] = Uw[1]; u[2] = Uw[2];
        } else {
            continue;
        }
        const float t = u[0] * lX.x + u[1] * lX.y + u[2] * lX.z + lf[0] * F.x + lf[1] * F.y + lf[2] * F.z;
        for (int k = 0; k < 3; k++) {
            lF[k] += s.w[q] * lf[k];
            g[k] += s.gw[q][k] * t;
        }
    }
    a.lx[i] = make_float4(lX.x + g[0], lX.y + g[1], lX.z + g[2], 0.f);
    a.lF[i] = make_float4(lF[0], lF[1], lF[2], 0.f);
    // the parts of F: Skalak, volume kv dV, bending (the rest)
    const int m = d.vcap[i];
    const CapDev cp = d.cap[m];
    const float kv = volume_factor(d, m);
    const float4 fs = d.Fsk[i], dv = d.dV[i];
    const float Fb[3] = {F.x - fs.x - kv * dv.x, F.y - fs.y - kv * dv.y, F.z - fs.z - kv * dv.z};
    // per-capsule FP64 sums (atomic: their order, and so their last bits, vary from run to run): lambda_F . dV
    // of the step for the volume transpose, and the parameter gradients, added over the steps (dF/dkS = F_Skalak
    // / kS, and likewise for bending and volume)
    const float ps = lF[0] * fs.x + lF[1] * fs.y + lF[2] * fs.z;
    const float pb = lF[0] * Fb[0] + lF[1] * Fb[1] + lF[2] * Fb[2];
    const float pd = lF[0] * dv.x + lF[1] * dv.y + lF[2] * dv.z;
    atomicAdd(a.capd + 4 * m + 3, (double)pd);
    if (cp.kS != 0.f) atomicAdd(a.capd + 4 * m + 0, (double)ps / cp.kS);
    if (cp.kB != 0.f) atomicAdd(a.capd + 4 * m + 1, (double)pb / cp.kB);
    if (cp.kV != 0.f) atomicAdd(a.capd + 4 * m + 2, (double)(kv * pd) / cp.kV);
    // bending, reversed from the force F_b = fb n with fb = 2 kB [2H(H^2 - K_G) + lap] A (Eq. 10)
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (cp.kB != 0.f) {
        const float4 nrm = d.nrm[i];
        const float2 AK = d.AK[i];
        const float A = AK.x, KG = AK.y, H = nrm.w;
        const float c2 = 2.f * cp.kB;
        const float fb = Fb[0] * nrm.x + Fb[1] * nrm.y + Fb[2] * nrm.z;
        const float lap = fb / (c2 * A) - 2.f * H * (H * H - KG);
        const float lfb = lF[0] * nrm.x + lF[1] * nrm.y + lF[2] * nrm.z;
        const float llap = lfb * c2 * A;
        float lH = lfb * c2 * A * (6.f * H * H - 2.f * KG);
        const float lKG = -lfb * c2 * A * 2.f * H;
        const float lA = lfb * c2 * (2.f * H * (H * H - KG) + lap) - lap / A * llap;
        const float mu = 0.5f * llap / A;              // adjoint of the cotangent sum of the Laplace-Beltrami
        float csum = 0.f;
        for (int qq = d.vt_off[i]; qq < d.vt_off[i + 1]; qq++) {
            const float2 ct = d.ccot[d.vt_idx[qq]];
            csum += ct.x + ct.y;
        }
        lH -= mu * csum;
        r0 = make_float4(mu, lH, lKG, lA);
        r1 = make_float4(fb * lF[0], fb * lF[1], fb * lF[2], H);
    }
    a.vb0[i] = r0;
    a.vb1[i] = r1;
}

// Per vertex: the second reverse stage of bending -- H's adjoint gathers the neighbours' Laplace-Beltrami terms,
// then the chain rule through H = K . n / 2, K = Ksum / (2A), n = Nsum / |Nsum|, K_G = (2 pi - angles) / A.
__global__ void k_cap_adj_vert2(DevState d, AdjCap a) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.NV) return;
    const CapDev cp = d.cap[d.vcap[i]];
    if (cp.kB == 0.f) {
        a.va[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        a.vK[i] = a.va[i];
        a.vN[i] = a.va[i];
        return;
    }
    const float4 r0 = a.vb0[i], r1 = a.vb1[i];
    float lH = r0.y;
    float3 Ks = make_float3(0.f, 0.f, 0.f), Ns = Ks;
    for (int qq = d.vt_off[i]; qq < d.vt_off[i + 1]; qq++) {
        const int c = d.vt_idx[qq];
        const int2 nb = d.cnb[c];
        const float2 ct = d.ccot[c];                   // (cot at j, cot at l); edge (i, j) carries cot at l
        lH += a.vb0[nb.x].x * ct.y + a.vb0[nb.y].x * ct.x;
        const float4 kc = d.corner[4 * c + 2], nc = d.corner[4 * c + 3];
        Ks.x += kc.x; Ks.y += kc.y; Ks.z += kc.z;
        Ns.x += nc.x; Ns.y += nc.y; Ns.z += nc.z;
    }
    const float4 nrm = d.nrm[i];
    const float2 AK = d.AK[i];
    const float A = AK.x, KG = AK.y;
    const float hA = 0.5f / A;
    const float K[3] = {hA * Ks.x, hA * Ks.y, hA * Ks.z};
    const float n[3] = {nrm.x, nrm.y, nrm.z};
    float lK[3], ln[3];
    for (int k = 0; k < 3; k++) {
        lK[k] = 0.5f * n[k] * lH;
        ln[k] = (k == 0 ? r1.x : (k == 1 ? r1.y : r1.z)) + 0.5f * K[k] * lH;
    }
    float lA = r0.w - (K[0] * lK[0] + K[1] * lK[1] + K[2] * lK[2]) / A - KG * r0.z / A;
    const float lang = -r0.z / A;
    const float inv = rsqrtf(Ns.x * Ns.x + Ns.y * Ns.y + Ns.z * Ns.z);
    const float lnn = ln[0] * n[0] + ln[1] * n[1] + ln[2] * n[2];
    a.va[i] = make_float4(lA, lang, r0.x, r1.w);        // (lambda_A, lambda_angle, mu, H)
    a.vK[i] = make_float4(hA * lK[0], hA * lK[1], hA * lK[2], 0.f);
    a.vN[i] = make_float4((ln[0] - lnn * n[0]) * inv, (ln[1] - lnn * n[1]) * inv, (ln[2] - lnn * n[2]) * inv, 0.f);
}

// Per triangle: the forward triangle pass (Skalak corner forces, volume records, bending records) with dual
// numbers over the 9 coordinates, contracted with the adjoints of everything it feeds: lambda_F of the corner
// forces, kv lambda_F of the volume records, and the bending stages' adjoints of the mixed-area shares, angles,
// mean-curvature vectors, face normal and cotangents.  Writes lambda . d/dP per corner.
__global__ void k_cap_adj_tri(DevState d, AdjCap a) {
    pdl_wait();
    pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= d.NT) return;
    const int4 T = d.tri[t];
    const CapDev cp = d.cap[T.w];
    const float4 R = d.tref[t];
    const float4 r0f = d.X[cp.v0];
    const int vid[3] = {T.x, T.y, T.z};
    V9 P[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float4 x = d.X[vid[k]];
        P[k] = {dc(x.x), dc(x.y), dc(x.z)};
        P[k].x.d[3 * k] = 1.f;
        P[k].y.d[3 * k + 1] = 1.f;
        P[k].z.d[3 * k + 2] = 1.f;
    }
    const V9 r0 = {dc(r0f.x), dc(r0f.y), dc(r0f.z)};
    float gacc[9];
#pragma unroll
    for (int k = 0; k < 9; k++) gacc[k] = 0.f;
    const float kv = volume_factor(d, T.w);
    float4 lF[3];
#pragma unroll
    for (int k = 0; k < 3; k++) lF[k] = a.lF[vid[k]];
    // ---- Skalak (Eq. 6, 8), as the forward triangle pass computes it
    {
        const V9 e1 = P[1] - P[0], e2 = P[2] - P[0];
        const D9 g11 = vdot(e1, e1), g12 = vdot(e1, e2), g22 = vdot(e2, e2);
        const float idet0 = R.x * R.z - R.y * R.y;
        const D9 I1 = R.x * g11 + (2.f * R.y) * g12 + R.z * g22 + (-2.f);
        const D9 I2 = idet0 * (g11 * g22 - g12 * g12) + (-1.f);
        const float pre = 0.25f * cp.kS * R.w;
        const D9 d1 = pre * (2.f * I1 + 2.f), d2 = pre * ((2.f * cp.C) * I2 + (-2.f));
        const D9 W11 = R.x * d1 + idet0 * (d2 * g22);
        const D9 W12 = (2.f * R.y) * d1 - (2.f * idet0) * (d2 * g12);
        const D9 W22 = R.z * d1 + idet0 * (d2 * g11);
        const V9 G1 = (2.f * W11) * e1 + W12 * e2;
        const V9 G2 = W12 * e1 + (2.f * W22) * e2;
        const V9 Fc[3] = {G1 + G2, -1.f * G1, -1.f * G2};
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int q = 0; q < 9; q++) gacc[q] += vcon(lF[k], Fc[k], q);
    }
    // ---- volume records dV_k = (P_j - r0) x (P_l - r0) / 6 (Eq. 7), weighted by kv
    if (kv != 0.f) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const V9 dv = (1.f / 6.f) * vcross(P[(k + 1) % 3] - r0, P[(k + 2) % 3] - r0);
            const float4 l = make_float4(kv * lF[k].x, kv * lF[k].y, kv * lF[k].z, 0.f);
#pragma unroll
            for (int q = 0; q < 9; q++) gacc[q] += vcon(l, dv, q);
        }
    }
    // ---- bending records (Meyer operators, Eq. 9-10)
    if (cp.kB != 0.f) {
        float4 va[3], vK[3], vN = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            va[k] = a.va[vid[k]];
            vK[k] = a.vK[vid[k]];
            const float4 n = a.vN[vid[k]];
            vN.x += n.x; vN.y += n.y; vN.z += n.z;
        }
        const V9 e1 = P[1] - P[0], e2 = P[2] - P[0];
        const V9 nrm = vcross(e1, e2);
        const D9 s2 = dsqrt(vdot(nrm, nrm));
        const D9 area = 0.5f * s2;
        D9 dots[3], cots[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            dots[k] = vdot(P[(k + 1) % 3] - P[k], P[(k + 2) % 3] - P[k]);
            cots[k] = dots[k] / s2;
        }
        const int obtuse = dots[0].v < 0.f ? 0 : (dots[1].v < 0.f ? 1 : (dots[2].v < 0.f ? 2 : -1));
#pragma unroll
        for (int q = 0; q < 9; q++) gacc[q] += vcon(vN, nrm, q);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int j = (k + 1) % 3, l = (k + 2) % 3;
            const V9 aij = P[j] - P[k], ail = P[l] - P[k];
            const V9 K = (-1.f * cots[l]) * aij + (-1.f * cots[j]) * ail;
            D9 Ash;
            if (obtuse < 0) Ash = 0.125f * (cots[l] * vdot(aij, aij) + cots[j] * vdot(ail, ail));
            else Ash = (obtuse == k ? 0.5f : 0.25f) * area;
            const D9 th = datan2(s2, dots[k]);
            // cotangent of the angle at k: used by the Laplace-Beltrami of the two other corners
            const float lcot = (va[j].z - va[l].z) * (va[l].w - va[j].w);
#pragma unroll
            for (int q = 0; q < 9; q++)
                gacc[q] += va[k].x * Ash.d[q] + va[k].y * th.d[q] + vcon(vK[k], K, q) + lcot * cots[k].d[q];
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) a.lp[3 * t + k] = make_float4(gacc[3 * k], gacc[3 * k + 1], gacc[3 * k + 2], 0.f);
}

// Per vertex: lambda_X += its corners' contributions and the volume factor's (d kv / dX = -kV / V0 dV); then the
// fields of the step are cleared at its stencil's fluid nodes (spread force and marks, luh, lfi, uh), which no
// vertex's gather reads.
__global__ void k_cap_adj_gather(LbmParams p, DevState d, AdjCap a) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.NV) return;
    float4 l = a.lx[i];
    for (int qq = d.vt_off[i]; qq < d.vt_off[i + 1]; qq++) {
        const float4 g = a.lp[d.vt_idx[qq]];
        l.x += g.x; l.y += g.y; l.z += g.z;
    }
    const int m = d.vcap[i];
    const CapDev c = d.cap[m];
    const float s = (float)(-(double)c.kV / c.V0 * a.capd[4 * m + 3]);
    const float4 dv = d.dV[i];
    l.x += s * dv.x; l.y += s * dv.y; l.z += s * dv.z;
    a.lx[i] = l;
    const AdjStencil st = adj_stencil(p, d.X[i]);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if (!st.fluid[q]) continue;
        const unsigned int n = st.node[q];
        for (int k = 0; k < 3; k++) {
            d.Fibm[(size_t)k * p.N + n] = 0ull;
            a.luh[(size_t)k * p.N + n] = 0.f;
            a.lfi[(size_t)k * p.N + n] = 0.f;
            a.uh[(size_t)k * p.N + n] = 0.f;
        }
        d.mask[n >> 5] = 0u;
    }
}

void launch_cap_adj_spread(const LbmParams& p, const DevState& d, const AdjCap& a, cudaStream_t st) {
    launch_k(k_cap_adj_spread, dim3((d.NV + 127) / 128), dim3(128), 0, st, p, d, a);
}

void launch_cap_adj_vertices(const LbmParams& p, const DevState& d, const AdjCap& a, cudaStream_t st) {
    const int b = 128;
    launch_k(k_cap_adj_vert, dim3((d.NV + b - 1) / b), dim3(b), 0, st, p, d, a);
    launch_k(k_cap_adj_vert2, dim3((d.NV + b - 1) / b), dim3(b), 0, st, d, a);
    launch_k(k_cap_adj_tri, dim3((d.NT + 63) / 64), dim3(64), 0, st, d, a);
    launch_k(k_cap_adj_gather, dim3((d.NV + b - 1) / b), dim3(b), 0, st, p, d, a);
}

}  // namespace scbb
