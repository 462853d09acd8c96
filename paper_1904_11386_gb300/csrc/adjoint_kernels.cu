// Adjoint kernels of the periodic two-component fluid step (the passes are described in adjoint.cuh).
#include <math.h>

#include "adjoint.cuh"

namespace scbb {

namespace {

constexpr int ADJ_THREADS = 256;

// Node of the periodic lattice at (x + dx, y + dy, z + dz).
__device__ __forceinline__ unsigned int pnode(const LbmParams& p, int x, int y, int z, int dx, int dy, int dz) {
    return (unsigned)wrapi(x + dx, p.nx) + (unsigned)p.nx * ((unsigned)wrapi(y + dy, p.ny) +
                                                             (unsigned)p.ny * (unsigned)wrapi(z + dz, p.nz));
}

__device__ __forceinline__ float dpsi_fn(float rho, int kind) { return kind == 1 ? 1.f : expf(-rho); }

}  // namespace

int adj_blocks(const LbmParams& p) {
    const long long need = ((long long)p.N + ADJ_THREADS - 1) / ADJ_THREADS;
    return (int)(need < 152 * 8 ? need : 152 * 8);
}

__global__ void __launch_bounds__(ADJ_THREADS) k_adj_final(LbmParams p, const float* __restrict__ gA,
                                                           const float* __restrict__ gB, float* __restrict__ lam) {
    const unsigned int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= p.N) return;
    const int z = y / p.nxy, r = y - z * p.nxy, yy = r / p.nx, x = r - yy * p.nx;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const unsigned int m = pnode(p, x, yy, z, dir_x(i), dir_y(i), dir_z(i));
        lam[(size_t)i * p.N + y] = gA[m];
        lam[(size_t)(Q + i) * p.N + y] = gB[m];
    }
}

// Local pass (one thread per node, grid-stride over a fixed grid).
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_local(LbmParams p, const float* __restrict__ S,
                                                           const float* __restrict__ rho,
                                                           const float* __restrict__ lam, float* __restrict__ scr,
                                                           double* __restrict__ part) {
    float acc[ADJ_PARAMS] = {0.f, 0.f, 0.f, 0.f};
    const size_t N = p.N;
    for (unsigned int n = blockIdx.x * blockDim.x + threadIdx.x; n < p.N; n += gridDim.x * blockDim.x) {
        const int z = n / p.nxy, r = n - z * p.nxy, y = r / p.nx, x = r - y * p.nx;
        // forward quantities of the node (Eq. 1-5, 13)
        float jx = 0.f, jy = 0.f, jz = 0.f;
        float sA[3] = {0.f, 0.f, 0.f}, sB[3] = {0.f, 0.f, 0.f};   // sum_i w_i psi^{B|A}(x + c_i) c_i
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const unsigned int src = pnode(p, x, y, z, -dir_x(i), -dir_y(i), -dir_z(i));
            const float f = S[(size_t)i * N + src] + S[(size_t)(Q + i) * N + src];
            jx += dir_x(i) * f;
            jy += dir_y(i) * f;
            jz += dir_z(i) * f;
            if (i > 0) {
                const unsigned int m = pnode(p, x, y, z, dir_x(i), dir_y(i), dir_z(i));
                const float wpB = dir_w(i) * psi_fn(rho[N + m], p.psi_kind);
                const float wpA = dir_w(i) * psi_fn(rho[m], p.psi_kind);
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
        const float uA[3] = {up[0] + ta * FA[0], up[1] + ta * FA[1], up[2] + ta * FA[2]};
        const float uB[3] = {up[0] + tb * FB[0], up[1] + tb * FB[1], up[2] + tb * FB[2]};
        const float uuA = uA[0] * uA[0] + uA[1] * uA[1] + uA[2] * uA[2];
        const float uuB = uB[0] * uB[0] + uB[1] * uB[1] + uB[2] * uB[2];
        // adjoint of f* = f + omega (f_eq(rho, u) - f) through f_eq:
        //   d f_eq,i / d rho = w_i (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u)
        //   d f_eq,i / d u   = w_i rho (3 c_i + 9 (c_i.u) c_i - 3 u)
        float arA = 0.f, arB = 0.f;
        float auA[3] = {0.f, 0.f, 0.f}, auB[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const float a = lam[(size_t)i * N + n], b = lam[(size_t)(Q + i) * N + n];
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
        // rho^c: through f_eq, through tau F^c / rho^c, through rho^c g, through u' = j / rho_t
        const float rA = arA - (ra > 0.f ? (aFA[0] * FA[0] + aFA[1] * FA[1] + aFA[2] * FA[2]) / ra : 0.f) +
                   (aFA[0] * p.g[0] + aFA[1] * p.g[1] + aFA[2] * p.g[2]) - aupu * irt;
        const float rB = arB - (rb > 0.f ? (aFB[0] * FB[0] + aFB[1] * FB[1] + aFB[2] * FB[2]) / rb : 0.f) +
                   (aFB[0] * p.g[0] + aFB[1] * p.g[1] + aFB[2] * p.g[2]) - aupu * irt;
        const float gpA = -p.G * (aFA[0] * sA[0] + aFA[1] * sA[1] + aFA[2] * sA[2]);
        const float gpB = -p.G * (aFB[0] * sB[0] + aFB[1] * sB[1] + aFB[2] * sB[2]);
        float* o = scr + n;
        o[0 * N] = rA;
        o[1 * N] = rB;
        o[2 * N] = aup[0] * irt;
        o[3 * N] = aup[1] * irt;
        o[4 * N] = aup[2] * irt;
        o[5 * N] = gpA;
        o[6 * N] = gpB;
        for (int k = 0; k < 3; k++) {
            o[(7 + k) * N] = p.G * pa * aFA[k];
            o[(10 + k) * N] = p.G * pb * aFB[k];
        }
        // dL/dG = sum_c -psi^c (dL/dF^c . s^c);  dL/dg = sum_c rho^c dL/dF^c
        acc[0] -= pa * (aFA[0] * sA[0] + aFA[1] * sA[1] + aFA[2] * sA[2]) +
                  pb * (aFB[0] * sB[0] + aFB[1] * sB[1] + aFB[2] * sB[2]);
        for (int k = 0; k < 3; k++) acc[1 + k] += ra * aFA[k] + rb * aFB[k];
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

// Push pass (one thread per node y).
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_push(LbmParams p, const float* __restrict__ rho,
                                                          const float* __restrict__ lam_in,
                                                          const float* __restrict__ scr,
                                                          float* __restrict__ lam_out) {
    const unsigned int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= p.N) return;
    const size_t N = p.N;
    const int z = y / p.nxy, r = y - z * p.nxy, yy = r / p.nx, x = r - yy * p.nx;
    // transposed pseudo-potential stencil: psi^A(y) enters F^B(y - c_i) with weight w_i c_i, and vice versa
    float apA = scr[5 * N + y], apB = scr[6 * N + y];
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const unsigned int m = pnode(p, x, yy, z, -dir_x(i), -dir_y(i), -dir_z(i));
        const float bBx = scr[10 * N + m], bBy = scr[11 * N + m], bBz = scr[12 * N + m];
        const float bAx = scr[7 * N + m], bAy = scr[8 * N + m], bAz = scr[9 * N + m];
        apA -= dir_w(i) * (dir_x(i) * bBx + dir_y(i) * bBy + dir_z(i) * bBz);
        apB -= dir_w(i) * (dir_x(i) * bAx + dir_y(i) * bAy + dir_z(i) * bAz);
    }
    const float aRA = scr[y] + dpsi_fn(rho[y], p.psi_kind) * apA;
    const float aRB = scr[N + y] + dpsi_fn(rho[N + y], p.psi_kind) * apB;
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
        const unsigned int src = pnode(p, x, yy, z, -dir_x(i), -dir_y(i), -dir_z(i));
        lam_out[(size_t)i * N + src] = gA;
        lam_out[(size_t)(Q + i) * N + src] = gB;
    }
}

__global__ void __launch_bounds__(ADJ_THREADS) k_adj_initial(LbmParams p, const float* __restrict__ S0,
                                                             const float* __restrict__ lam0,
                                                             float* __restrict__ drho) {
    const unsigned int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.N) return;
    const size_t N = p.N;
    const int z = x / p.nxy, r = x - z * p.nxy, y = r / p.nx, xx = r - y * p.nx;
    float ra = 0.f, rb = 0.f, da = 0.f, db = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const unsigned int src = pnode(p, xx, y, z, -dir_x(i), -dir_y(i), -dir_z(i));
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
    k_adj_final<<<(p.N + ADJ_THREADS - 1) / ADJ_THREADS, ADJ_THREADS, 0, st>>>(p, gA, gB, lam);
}

void launch_adj_step(const LbmParams& p, const float* S, const float* rho, const float* lam_in, float* lam_out,
                     float* scr, double* part, cudaStream_t st) {
    k_adj_local<<<adj_blocks(p), ADJ_THREADS, 0, st>>>(p, S, rho, lam_in, scr, part);
    k_adj_push<<<(p.N + ADJ_THREADS - 1) / ADJ_THREADS, ADJ_THREADS, 0, st>>>(p, rho, lam_in, scr, lam_out);
}

void launch_adj_initial(const LbmParams& p, const float* S0, const float* lam0, float* drho, cudaStream_t st) {
    k_adj_initial<<<(p.N + ADJ_THREADS - 1) / ADJ_THREADS, ADJ_THREADS, 0, st>>>(p, S0, lam0, drho);
}

}  // namespace scbb
