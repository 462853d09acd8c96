// Adjoint kernels of the periodic two-component fluid step (the passes are described in adjoint.cuh).
#include <math.h>

#include "adjoint.cuh"
#include "pdl.cuh"

namespace scbb {

namespace {

constexpr int ADJ_THREADS = 256;

// Node at (x + dx, y + dy, z + dz): x and y periodic, z periodic without walls (with walls the callers keep
// z + dz inside 0 .. nz-1).  The kernels are instantiated with and without walls (W), so that the periodic
// box compiles without the wall branches.
template <bool W>
__device__ __forceinline__ unsigned int pnode(const LbmParams& p, int x, int y, int z, int dx, int dy, int dz) {
    const int zz = W ? z + dz : wrapi(z + dz, p.nz);
    return (unsigned)wrapi(x + dx, p.nx) + (unsigned)p.nx * ((unsigned)wrapi(y + dy, p.ny) + (unsigned)p.ny * zz);
}

template <bool W>
__device__ __forceinline__ bool fluid_z(const LbmParams& p, int z) {
    return W ? (z >= 1 && z <= p.nz - 2) : true;
}

__device__ __forceinline__ float dpsi_fn(float rho, int kind) { return kind == 1 ? 1.f : expf(-rho); }

}  // namespace

int adj_blocks(const LbmParams& p) {
    const long long need = ((long long)p.N + ADJ_THREADS - 1) / ADJ_THREADS;
    return (int)(need < 152 * 8 ? need : 152 * 8);
}

template <bool W>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_final(LbmParams p, const float* __restrict__ gA,
                                                           const float* __restrict__ gB, float* __restrict__ lam) {
    const unsigned int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= p.N) return;
    const int z = y / p.nxy, r = y - z * p.nxy, yy = r / p.nx, x = r - yy * p.nx;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        // the slot feeds the density of the node it streams to; with walls only fluid nodes have one
        float a = 0.f, b = 0.f;
        if (fluid_z<W>(p, z + dir_z(i))) {
            const unsigned int m = pnode<W>(p, x, yy, z, dir_x(i), dir_y(i), dir_z(i));
            a = gA[m];
            b = gB[m];
        }
        lam[(size_t)i * p.N + y] = a;
        lam[(size_t)(Q + i) * p.N + y] = b;
    }
}

// Local pass (one thread per node, grid-stride over a fixed grid).  IB: the step carried the spread force of a
// 2-point immersed boundary (ib.Fibm at the nodes marked in ib.mask) and wrote the half-force velocity there; ib.luh
// holds the adjoint of that velocity, and the pass writes the adjoint of the spread force (ib.lfi) and the
// half-force velocity itself (ib.uh) at the marked nodes.
template <bool W, bool IB>
__global__ void __launch_bounds__(ADJ_THREADS, 3) k_adj_local(LbmParams p, const float* __restrict__ S,
                                                           const float* __restrict__ rho,
                                                           const float* __restrict__ ghost,
                                                           const float* __restrict__ lam, float* __restrict__ scr,
                                                           double* __restrict__ part, AdjIB ib) {
    pdl_wait();
    float acc[ADJ_PARAMS] = {0.f, 0.f, 0.f, 0.f};
    const size_t N = p.N;
    for (unsigned int n = blockIdx.x * blockDim.x + threadIdx.x; n < p.N; n += gridDim.x * blockDim.x) {
        const int z = n / p.nxy, r = n - z * p.nxy, y = r / p.nx, x = r - y * p.nx;
        if (!fluid_z<W>(p, z)) {                 // wall node: no collision, nothing to send
#pragma unroll
            for (int k = 0; k < ADJ_SCR; k++) scr[(size_t)k * N + n] = 0.f;
            continue;
        }
        // forward quantities of the node (Eq. 1-5, 13)
        float jx = 0.f, jy = 0.f, jz = 0.f;
        float sA[3] = {0.f, 0.f, 0.f}, sB[3] = {0.f, 0.f, 0.f};   // sum_i w_i psi^{B|A}(x + c_i) c_i
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const unsigned int src = pnode<W>(p, x, y, z, -dir_x(i), -dir_y(i), -dir_z(i));
            const float f = S[(size_t)i * N + src] + S[(size_t)(Q + i) * N + src];
            jx += dir_x(i) * f;
            jy += dir_y(i) * f;
            jz += dir_z(i) * f;
            if (i > 0) {
                // psi of the neighbour: its density, or on a wall plane the wall's virtual density
                float nA, nB;
                if (fluid_z<W>(p, z + dir_z(i))) {
                    const unsigned int m = pnode<W>(p, x, y, z, dir_x(i), dir_y(i), dir_z(i));
                    nA = rho[m];
                    nB = rho[N + m];
                } else {
                    const int w = z + dir_z(i) == 0 ? 0 : 1;
                    const unsigned int rm = (unsigned)wrapi(x + dir_x(i), p.nx) + (unsigned)p.nx * wrapi(y + dir_y(i), p.ny);
                    nA = ghost[(size_t)(w * 2 + 0) * p.nxy + rm];
                    nB = ghost[(size_t)(w * 2 + 1) * p.nxy + rm];
                }
                const float wpB = dir_w(i) * psi_fn(nB, p.psi_kind);
                const float wpA = dir_w(i) * psi_fn(nA, p.psi_kind);
                sA[0] += wpB * dir_x(i); sA[1] += wpB * dir_y(i); sA[2] += wpB * dir_z(i);
                sB[0] += wpA * dir_x(i); sB[1] += wpA * dir_y(i); sB[2] += wpA * dir_z(i);
            }
        }
        const float ra = rho[n], rb = rho[N + n];
        const float pa = psi_fn(ra, p.psi_kind), pb = psi_fn(rb, p.psi_kind);
        float FA[3], FB[3];
        for (int k = 0; k < 3; k++) {
            FA[k] = -pa * p.G * sA[k] + ra * p.g[k];
            FB[k] = -pb * p.G * sB[k] + rb * p.g[k];
        }
        const float rt = ra + rb, irt = 1.f / rt;
        const float up[3] = {jx * irt, jy * irt, jz * irt};
        const float ta = ra > 0.f ? p.tau / ra : 0.f, tb = rb > 0.f ? p.tau / rb : 0.f;
        // spread force (its share rho^c / rho on component c shifts both velocities by tau Fi / rho)
        bool marked = false;
        float Fi[3] = {0.f, 0.f, 0.f};
        if (IB) {
            marked = (ib.mask[n >> 5] >> (n & 31)) & 1u;
            if (marked)
                for (int k = 0; k < 3; k++) Fi[k] = ibm_unfix(ib.Fibm[(size_t)k * N + n]);
        }
        const float tf = p.tau * irt;
        const float uA[3] = {up[0] + ta * FA[0] + tf * Fi[0], up[1] + ta * FA[1] + tf * Fi[1],
                             up[2] + ta * FA[2] + tf * Fi[2]};
        const float uB[3] = {up[0] + tb * FB[0] + tf * Fi[0], up[1] + tb * FB[1] + tf * Fi[1],
                             up[2] + tb * FB[2] + tf * Fi[2]};
        const float uuA = uA[0] * uA[0] + uA[1] * uA[1] + uA[2] * uA[2];
        const float uuB = uB[0] * uB[0] + uB[1] * uB[1] + uB[2] * uB[2];
        // adjoint of f* = f + omega (f_eq(rho, u) - f) through f_eq:
        //   d f_eq,i / d rho = w_i (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u)
        //   d f_eq,i / d u   = w_i rho (3 c_i + 9 (c_i.u) c_i - 3 u)
        float arA = 0.f, arB = 0.f;
        float auA[3] = {0.f, 0.f, 0.f}, auB[3] = {0.f, 0.f, 0.f};
        float wallA = 0.f, wallB = 0.f;       // moving-wall term of the bounced values (Eq. 11)
#pragma unroll
        for (int i = 0; i < Q; i++) {
            // adjoint of f*_i: where f*_i stays in the fluid its own slot; where c_i points into a wall, the slot
            // of the wall node its bounced value -6 w_i c_i.U rho was stored in (the node pulls it back)
            float a, b;
            if (fluid_z<W>(p, z + dir_z(i))) {
                a = lam[(size_t)i * N + n];
                b = lam[(size_t)(Q + i) * N + n];
            } else {
                const unsigned int m = pnode<W>(p, x, y, z, dir_x(i), dir_y(i), dir_z(i));
                a = lam[(size_t)dir_opp(i) * N + m];
                b = lam[(size_t)(Q + dir_opp(i)) * N + m];
                const float* U = z + dir_z(i) == 0 ? p.ulo : p.uhi;
                const float cU = 6.f * dir_w(i) * (dir_x(i) * U[0] + dir_y(i) * U[1] + dir_z(i) * U[2]);
                wallA -= cU * a;
                wallB -= cU * b;
            }
            const float cuA = dir_x(i) * uA[0] + dir_y(i) * uA[1] + dir_z(i) * uA[2];
            const float cuB = dir_x(i) * uB[0] + dir_y(i) * uB[1] + dir_z(i) * uB[2];
            arA += a * dir_w(i) * (1.f + 3.f * cuA + 4.5f * cuA * cuA - 1.5f * uuA);
            arB += b * dir_w(i) * (1.f + 3.f * cuB + 4.5f * cuB * cuB - 1.5f * uuB);
            const float qa = a * dir_w(i) * ra, qb = b * dir_w(i) * rb;
            const float c3[3] = {(float)dir_x(i), (float)dir_y(i), (float)dir_z(i)};
            for (int k = 0; k < 3; k++) {
                auA[k] += qa * (3.f * c3[k] + 9.f * cuA * c3[k] - 3.f * uA[k]);
                auB[k] += qb * (3.f * c3[k] + 9.f * cuB * c3[k] - 3.f * uB[k]);
            }
        }
        const float om = p.omega;
        arA *= om; arB *= om;
        float aup[3], aFA[3], aFB[3];
        for (int k = 0; k < 3; k++) {
            auA[k] *= om;
            auB[k] *= om;
            aup[k] = auA[k] + auB[k];         // u^c = u' + tau F^c / rho^c
            aFA[k] = ta * auA[k];
            aFB[k] = tb * auB[k];
        }
        const float aupu = aup[0] * up[0] + aup[1] * up[1] + aup[2] * up[2];
        // immersed boundary: the half-force velocity uh = (j + (F^A + F^B + Fi) / 2) / rho_t (Eq. 5) at a marked
        // node, with F^c = F_SC^c + rho^c g: its adjoint luh reaches j, both Shan-Chen forces and Fi with
        // 1 / rho_t, 1 / (2 rho_t), 1 / (2 rho_t), g with 1/2, and rho^c with (g/2 - uh) / rho_t
        float luh[3] = {0.f, 0.f, 0.f}, rib = 0.f;
        if (IB && marked) {
            float uh[3];
            for (int k = 0; k < 3; k++) {
                luh[k] = ib.luh[(size_t)k * N + n];
                uh[k] = (k == 0 ? jx : (k == 1 ? jy : jz)) * irt + 0.5f * (FA[k] + FB[k] + Fi[k]) * irt;
                ib.uh[(size_t)k * N + n] = uh[k];
            }
            // tau Fi / rho_t in both velocities, and uh's 1 / rho_t (its rho^c g / 2 reaches rho^c through the
            // Shan-Chen force adjoints' g term below)
            rib = -tf * irt * (aup[0] * Fi[0] + aup[1] * Fi[1] + aup[2] * Fi[2]) -
                  irt * (luh[0] * uh[0] + luh[1] * uh[1] + luh[2] * uh[2]);
            for (int k = 0; k < 3; k++) ib.lfi[(size_t)k * N + n] = tf * aup[k] + 0.5f * irt * luh[k];
        }
        // the Shan-Chen forces' adjoints: through the velocities and, at marked nodes, through uh
        float sFA[3], sFB[3];
        for (int k = 0; k < 3; k++) {
            sFA[k] = aFA[k] + 0.5f * irt * luh[k];
            sFB[k] = aFB[k] + 0.5f * irt * luh[k];
        }
        // rho^c: through f_eq, through tau F^c / rho^c, through rho^c g, through u' = j / rho_t
        const float rA = arA - (ra > 0.f ? (aFA[0] * FA[0] + aFA[1] * FA[1] + aFA[2] * FA[2]) / ra : 0.f) +
                         (sFA[0] * p.g[0] + sFA[1] * p.g[1] + sFA[2] * p.g[2]) - aupu * irt + wallA + rib;
        const float rB = arB - (rb > 0.f ? (aFB[0] * FB[0] + aFB[1] * FB[1] + aFB[2] * FB[2]) / rb : 0.f) +
                         (sFB[0] * p.g[0] + sFB[1] * p.g[1] + sFB[2] * p.g[2]) - aupu * irt + wallB + rib;
        const float gpA = -p.G * (sFA[0] * sA[0] + sFA[1] * sA[1] + sFA[2] * sA[2]);
        const float gpB = -p.G * (sFB[0] * sB[0] + sFB[1] * sB[1] + sFB[2] * sB[2]);
        float* o = scr + n;
        o[0 * N] = rA;
        o[1 * N] = rB;
        o[2 * N] = (aup[0] + luh[0]) * irt;
        o[3 * N] = (aup[1] + luh[1]) * irt;
        o[4 * N] = (aup[2] + luh[2]) * irt;
        o[5 * N] = gpA;
        o[6 * N] = gpB;
        for (int k = 0; k < 3; k++) {
            o[(7 + k) * N] = p.G * pa * sFA[k];
            o[(10 + k) * N] = p.G * pb * sFB[k];
        }
        // dL/dG = sum_c -psi^c (dL/dF^c . s^c);  dL/dg = sum_c rho^c dL/dF^c (and uh's g/2)
        acc[0] -= pa * (sFA[0] * sA[0] + sFA[1] * sA[1] + sFA[2] * sA[2]) +
                  pb * (sFB[0] * sB[0] + sFB[1] * sB[1] + sFB[2] * sB[2]);
        for (int k = 0; k < 3; k++) acc[1 + k] += ra * aFA[k] + rb * aFB[k] + 0.5f * luh[k];
    }
    // block sums in a fixed order, added to this block's own slot
    __shared__ float sh[ADJ_PARAMS][ADJ_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < ADJ_PARAMS; k++) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < ADJ_PARAMS) {
        double s = 0.0;
        for (int q = 0; q < ADJ_THREADS / 32; q++) s += (double)sh[threadIdx.x][q];
        part[(size_t)blockIdx.x * ADJ_PARAMS + threadIdx.x] += s;
    }
}

// Wall pass (one thread per wall node w, both walls): the force at the fluid nodes next to the wall reads
// psi of the wall's virtual density; dL/dpsi gathers -w_i c_i . b(w - c_i) over those nodes, and gw holds
// dL/d(virtual density) = psi'(ghost) dL/dpsi, per wall and component.
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_wall(LbmParams p, const float* __restrict__ ghost,
                                                          const float* __restrict__ scr, float* __restrict__ gw) {
    pdl_wait();
    pdl_trigger();
    const unsigned int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2u * p.nxy) return;
    const size_t N = p.N;
    const int w = q / p.nxy, r = q - w * p.nxy, y = r / p.nx, x = r - y * p.nx;
    const int zw = w == 0 ? 0 : p.nz - 1, dz = w == 0 ? -1 : 1;     // c_z from the fluid plane into the wall
    float apA = 0.f, apB = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        if (dir_z(i) != dz) continue;
        const unsigned int m = pnode<true>(p, x, y, zw, -dir_x(i), -dir_y(i), -dir_z(i));
        apA -= dir_w(i) * (dir_x(i) * scr[10 * N + m] + dir_y(i) * scr[11 * N + m] + dir_z(i) * scr[12 * N + m]);
        apB -= dir_w(i) * (dir_x(i) * scr[7 * N + m] + dir_y(i) * scr[8 * N + m] + dir_z(i) * scr[9 * N + m]);
    }
    gw[(size_t)(w * 2 + 0) * p.nxy + r] = dpsi_fn(ghost[(size_t)(w * 2 + 0) * p.nxy + r], p.psi_kind) * apA;
    gw[(size_t)(w * 2 + 1) * p.nxy + r] = dpsi_fn(ghost[(size_t)(w * 2 + 1) * p.nxy + r], p.psi_kind) * apB;
}

// Push pass (one thread per node y).
template <bool W>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_push(LbmParams p, const float* __restrict__ rho,
                                                          const float* __restrict__ lam_in,
                                                          const float* __restrict__ scr,
                                                          const float* __restrict__ gw,
                                                          float* __restrict__ lam_out) {
    pdl_wait();
    const unsigned int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= p.N) return;
    const size_t N = p.N;
    const int z = y / p.nxy, r = y - z * p.nxy, yy = r / p.nx, x = r - yy * p.nx;
    if (!fluid_z<W>(p, z)) return;               // wall nodes pull nothing
    // transposed pseudo-potential stencil: psi^A(y) enters F^B(y - c_i) with weight w_i c_i, and vice versa
    float apA = scr[5 * N + y], apB = scr[6 * N + y];
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const unsigned int m = pnode<W>(p, x, yy, z, -dir_x(i), -dir_y(i), -dir_z(i));
        const float bBx = scr[10 * N + m], bBy = scr[11 * N + m], bBz = scr[12 * N + m];
        const float bAx = scr[7 * N + m], bAy = scr[8 * N + m], bAz = scr[9 * N + m];
        apA -= dir_w(i) * (dir_x(i) * bBx + dir_y(i) * bBy + dir_z(i) * bBz);
        apB -= dir_w(i) * (dir_x(i) * bAx + dir_y(i) * bAy + dir_z(i) * bAz);
    }
    float aRA = scr[y] + dpsi_fn(rho[y], p.psi_kind) * apA;
    float aRB = scr[N + y] + dpsi_fn(rho[N + y], p.psi_kind) * apB;
    if (W && (z == 1 || z == p.nz - 2)) {
        // a wall's virtual density is the mean density of the five fluid nodes (x, y), (x +- 1, y), (x, y +- 1)
        // of the plane next to it; this node is in the stencils of the same five wall nodes
        const int w = z == 1 ? 0 : 1;
        const float* ga = gw + (size_t)(w * 2 + 0) * p.nxy;
        const float* gb = gw + (size_t)(w * 2 + 1) * p.nxy;
        const int xm = wrapi(x - 1, p.nx), xp = wrapi(x + 1, p.nx);
        const int ym = wrapi(yy - 1, p.ny) * p.nx, y0 = yy * p.nx, yp = wrapi(yy + 1, p.ny) * p.nx;
        aRA += 0.2f * (ga[x + y0] + ga[xm + y0] + ga[xp + y0] + ga[x + ym] + ga[x + yp]);
        aRB += 0.2f * (gb[x + y0] + gb[xm + y0] + gb[xp + y0] + gb[x + ym] + gb[x + yp]);
    }
    const float Jx = scr[2 * N + y], Jy = scr[3 * N + y], Jz = scr[4 * N + y];
    const float keep = 1.f - p.omega;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const float cJ = dir_x(i) * Jx + dir_y(i) * Jy + dir_z(i) * Jz;
        float gA = aRA + cJ, gB = aRB + cJ;
        if (keep != 0.f) {
            gA += keep * lam_in[(size_t)i * N + y];
            gB += keep * lam_in[(size_t)(Q + i) * N + y];
        }
        const unsigned int src = pnode<W>(p, x, yy, z, -dir_x(i), -dir_y(i), -dir_z(i));
        lam_out[(size_t)i * N + src] = gA;
        lam_out[(size_t)(Q + i) * N + src] = gB;
    }
}

template <bool W>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_initial(LbmParams p, const float* __restrict__ S0,
                                                             const float* __restrict__ lam0,
                                                             float* __restrict__ drho) {
    const unsigned int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.N) return;
    const size_t N = p.N;
    const int z = x / p.nxy, r = x - z * p.nxy, y = r / p.nx, xx = r - y * p.nx;
    if (!fluid_z<W>(p, z)) {
        drho[x] = 0.f;
        drho[N + x] = 0.f;
        return;
    }
    float ra = 0.f, rb = 0.f, da = 0.f, db = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const unsigned int src = pnode<W>(p, xx, y, z, -dir_x(i), -dir_y(i), -dir_z(i));
        const float fa = S0[(size_t)i * N + src], fb = S0[(size_t)(Q + i) * N + src];
        ra += fa;
        rb += fb;
        da += lam0[(size_t)i * N + src] * fa;
        db += lam0[(size_t)(Q + i) * N + src] * fb;
    }
    drho[x] = ra > 0.f ? da / ra : 0.f;
    drho[N + x] = rb > 0.f ? db / rb : 0.f;
}

void launch_adj_final(const LbmParams& p, const float* gA, const float* gB, float* lam, cudaStream_t st) {
    const unsigned nb = (p.N + ADJ_THREADS - 1) / ADJ_THREADS;
    if (p.walls) k_adj_final<true><<<nb, ADJ_THREADS, 0, st>>>(p, gA, gB, lam);
    else k_adj_final<false><<<nb, ADJ_THREADS, 0, st>>>(p, gA, gB, lam);
}

void launch_adj_step(const LbmParams& p, const float* S, const float* rho, const float* ghost, const float* lam_in,
                     float* lam_out, float* scr, float* gw, double* part, cudaStream_t st, const AdjIB* ib) {
    const unsigned nb = (p.N + ADJ_THREADS - 1) / ADJ_THREADS;
    const AdjIB none{};
    const AdjIB& b = ib ? *ib : none;
    if (p.walls) {
        if (ib) launch_k(k_adj_local<true, true>, dim3(adj_blocks(p)), dim3(ADJ_THREADS), 0, st, p, S, rho, ghost, lam_in, scr, part, b);
        else launch_k(k_adj_local<true, false>, dim3(adj_blocks(p)), dim3(ADJ_THREADS), 0, st, p, S, rho, ghost, lam_in, scr, part, b);
        launch_k(k_adj_wall, dim3((2 * p.nxy + ADJ_THREADS - 1) / ADJ_THREADS), dim3(ADJ_THREADS), 0, st, p, ghost, scr, gw);
        launch_k(k_adj_push<true>, dim3(nb), dim3(ADJ_THREADS), 0, st, p, rho, lam_in, scr, gw, lam_out);
    } else {
        if (ib) launch_k(k_adj_local<false, true>, dim3(adj_blocks(p)), dim3(ADJ_THREADS), 0, st, p, S, rho, ghost, lam_in, scr, part, b);
        else launch_k(k_adj_local<false, false>, dim3(adj_blocks(p)), dim3(ADJ_THREADS), 0, st, p, S, rho, ghost, lam_in, scr, part, b);
        launch_k(k_adj_push<false>, dim3(nb), dim3(ADJ_THREADS), 0, st, p, rho, lam_in, scr, gw, lam_out);
    }
}

void launch_adj_initial(const LbmParams& p, const float* S0, const float* lam0, float* drho, cudaStream_t st) {
    const unsigned nb = (p.N + ADJ_THREADS - 1) / ADJ_THREADS;
    if (p.walls) k_adj_initial<true><<<nb, ADJ_THREADS, 0, st>>>(p, S0, lam0, drho);
    else k_adj_initial<false><<<nb, ADJ_THREADS, 0, st>>>(p, S0, lam0, drho);
}

}  // namespace scbb
