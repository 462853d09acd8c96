// Internal declarations shared by the CUDA translation units of libscbb (sm_103a).
//
// Population storage: two FP32 lattices S[c][i][N] (structure of arrays, x fastest).  A lattice holds the
// post-collision populations of the last step, not yet streamed; streaming is a pull, f_i(x) = S[i][x - c_i].
// Links that end on a wall node (Eq. 11) store the bounced value in the slot the receiving node pulls from,
// so every pull is the same plain gather and the density of any node can be recomputed from S.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/scbb.h"

namespace scbb {

constexpr int Q = 19;

// D3Q19 in the order rest, +x, -x, +y, -y, +z, -z, (+x+y), (-x-y), (+x-y), (-x+y), (+x+z), (-x-z), (+x-z),
// (-x+z), (+y+z), (-y-z), (+y-z), (-y+z); every direction is followed by its opposite.
__host__ __device__ constexpr int dir_x(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int dir_y(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int dir_z(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int dir_opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float dir_w(int i) {
    return i == 0 ? (1.0f / 3.0f) : (i <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}

// Lattice / fluid parameters passed by value to the fluid kernels.
struct LbmParams {
    int nx, ny, nz, nxy;
    unsigned int N;
    int walls;
    int zf0, zf1;           // fluid planes [zf0, zf1)
    int lz;                 // z-segment length of one bulk CTA
    float tau, omega, G;
    int psi_kind;
    float g[3];
    float ulo[3], uhi[3];
};

// One capsule's constants on the device.
struct CapDev {
    float kS, C, kB, kV, mass, colour;
    double V0;
    int v0, nv, t0, nt;
};

// Device-side buffers of a context (all carved from the caller's workspace).
struct DevState {
    float* S[2];            // populations, 2 * 19 * N floats each
    float* rho;             // [2][N] densities of the last collision
    float* u;               // [3][N] velocity incl. half force, written where the IBM mask is set
    float* Fibm;            // [3][N] spread immersed-boundary force density
    uint32_t* mask;         // [ceil(N/32)] IBM stencil bits
    float* wall_rho;        // [2 walls][2 comp][nxy] densities of the planes next to the walls
    float* ghost;           // [2 walls][2 comp][nxy] virtual densities of the wall planes
    double* red;            // reduction scratch
    int* err;               // sticky device error word
    // membranes
    int NV, NT, NM;
    float4* X;              // [NV] positions
    float4* V;              // [NV] velocities
    float4* F;              // [NV] total node force of the last step
    float4* Fsk;            // [NV] Skalak force
    float4* dV;             // [NV] volume gradient
    float4* nrm;            // [NV] unit normal (xyz) and H (w)
    float2* AK;             // [NV] mixed area, Gaussian curvature
    int4* tri;              // [NT] a, b, c, capsule
    float4* tref;           // [NT] inverse reference metric (ia, ib, ic) and reference area A0
    int* vt_off;            // [NV+1] vertex -> incident triangle CSR
    int* vt_idx;            // [3 NT] corner ids 3 * t + k of the triangles around each vertex
    int* vcap;              // [NV] capsule of each vertex
    CapDev* cap;            // [NM]
    double* cap_red;        // [NM][4] volume, centre of mass
    float4* corner;         // [3 NT][4] per-corner records of the membrane triangle pass (scratch)
    float2* ccot;           // [3 NT] cotangents of the angles at the two other corners j, l (scratch)
    float* tvol;            // [NT] volume term of each triangle (scratch)
    int2* cnb;              // [3 NT] global ids of the two other corners j, l (topology)
    float4* X0;             // [NV] initial shape (for resets)
};

// ---- launches (lbm_kernels.cu) ----
void launch_init_state(const LbmParams& p, float* S, const float* rho_st, const float* u_st, cudaStream_t st);
void launch_wall_ghost(const LbmParams& p, const float* S, float* wall_rho, float* ghost, cudaStream_t st);
void launch_bulk(const LbmParams& p, const float* S, float* D, float* rho, const float* ghost,
                 const float* Fibm, const uint32_t* mask, float* u, int* err, bool ibm, cudaStream_t st);
void launch_export(const LbmParams& p, const float* S, float* out, int what, cudaStream_t st);
void launch_moments_reduce(const LbmParams& p, const float* S, double* red, cudaStream_t st);
int bulk_grid_blocks(const LbmParams& p);

// ---- launches (membrane_kernels.cu) ----
void launch_capsule_reduce(const DevState& d, cudaStream_t st);
void launch_membrane_forces(const DevState& d, cudaStream_t st);
void launch_ibm_spread(const LbmParams& p, const DevState& d, cudaStream_t st);
void launch_ibm_interp(const LbmParams& p, const DevState& d, cudaStream_t st);
void launch_pp_forces(const LbmParams& p, const DevState& d, float eps, float d0, cudaStream_t st);

}  // namespace scbb
