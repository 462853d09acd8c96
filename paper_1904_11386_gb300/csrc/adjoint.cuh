// Reverse-mode derivative (adjoint) of the two-component fluid step, sm_103a.
//
// The forward step (Sec. II.A, II.D): pull f_i^c(x) = S^c[i][x - c_i]; rho^c, j; the
// Shan-Chen force F^c(x) = -psi^c(x) G sum_i w_i psi^c'(x + c_i) c_i + rho^c g (Eq. 13); the equilibrium
// velocity u^c = j / rho_t + tau F^c / rho^c; BGK f*_i^c = f_i^c + omega (f_eq,i(rho^c, u^c) - f_i^c) (Eq. 1-2),
// stored at S'^c[i][x]; next to a wall, a population leaving towards it is stored, bounced with the wall's
// velocity (Eq. 11), in the wall node's slot the node pulls back, and the force reads psi of the wall's virtual
// density (the mean density of five nodes of the first fluid plane).  Its adjoint maps lambda' = dL/dS' to
// lambda = dL/dS in two passes over the nodes (and, with walls, a pass over the wall nodes between them):
//
//   local   per node x: adjoints of rho^c, u^c, F^c, u', j from lambda'(x) (chain rule through f_eq and the
//           force), the local part of dL/dpsi^c(x), and b^c(x) = G psi^c(x) dL/dF^c(x), which the force at x
//           sends to psi^c' of the 18 neighbours; dL/dG and dL/dg accumulate per block
//   push    per node y: dL/dpsi^c(y) gathers -w_i c_i . b^c'(y - c_i) over the 18 neighbours (the transposed
//           pseudo-potential stencil), dL/drho^c(y) = local part + psi'(rho^c(y)) dL/dpsi^c(y), and
//           dL/df_i^c(y) = (1 - omega) lambda'^c[i][y] + dL/drho^c(y) + c_i . dL/dj(y) is pushed to
//           lambda^c[i][y - c_i] (the transpose of the pull)
//
// All arithmetic is FP32; the parameter gradients are FP32 per block and FP64 across blocks and steps.
#pragma once

#include "scbb_internal.cuh"

namespace scbb {

constexpr int ADJ_SCR = 13;        // per-node scratch: r^A, r^B, J[3], gpsi^A, gpsi^B, b^A[3], b^B[3]
constexpr int ADJ_PARAMS = 4;      // dL/dG, dL/dg[3]

// Blocks of the local pass: its grid is fixed so that each block adds its partial sums, in the same order
// every step, to its own slot of part[ADJ_PARAMS * adj_blocks(p)].
int adj_blocks(const LbmParams& p);

// lambda^c[i][y] = g^c(y + c_i): the adjoint of a lattice whose densities (after the pull) enter the loss
// with the weights g^c = dL/drho^c (device, N floats per component).
void launch_adj_final(const LbmParams& p, const float* gA, const float* gB, float* lam, cudaStream_t st);

// Immersed-boundary terms of a step (all [3][N] fields except mask): the spread force the step used and its
// marks, the adjoint of the half-force velocity it wrote at the marked nodes (in), the adjoint of the spread
// force and the half-force velocity itself at the marked nodes (out).
struct AdjIB {
    const IbmF* Fibm;
    const uint32_t* mask;
    const float* luh;
    float* lfi;
    float* uh;
};

// One step backwards: S is the lattice the forward step read, rho the densities it computed, ghost the wall
// planes' virtual densities it used (4 nxy floats, walls only), lam_in the adjoint of the lattice it wrote;
// writes lam_out, the adjoint of S.  scr holds ADJ_SCR * N floats, gw 4 nxy floats (walls only).  ib: the
// immersed-boundary terms of the step, or null.
void launch_adj_step(const LbmParams& p, const float* S, const float* rho, const float* ghost, const float* lam_in,
                     float* lam_out, float* scr, float* gw, double* part, cudaStream_t st, const AdjIB* ib = nullptr);

// ---- adjoint of a capsule coupled by the 2-point immersed boundary (adjoint_capsule.cu)
// Device buffers of the capsule's part of one backward step.
struct AdjCap {
    float4* lx;             // [NV] adjoint of the vertex positions (of X(t + 1) in, of X(t) out)
    float4* lF;             // [NV] adjoint of the node forces
    float4* vb0;            // [NV] bending, first reverse stage: (mu, lambda_H part, lambda_KG, lambda_A part)
    float4* vb1;            //      (fb lambda_F, H)
    float4* va;             // [NV] second stage: (lambda_A, lambda_angle sum, mu, H)
    float4* vK;             //      adjoint of the corner sum of mean-curvature vectors
    float4* vN;             //      adjoint of the corner sum of face normals
    float4* lp;             // [3 NT] per-corner contributions to lambda_X
    float* luh;             // [3][N] adjoint of the half-force velocity
    float* lfi;             // [3][N] adjoint of the spread force
    float* uh;              // [3][N] half-force velocity of the step
    double* capd;           // [4 NM] dL/dkS, dL/dkB, dL/dkV (summed over the steps), lambda_F . dV of the step
                            // (FP64 atomic sums of the vertex products)
};
// luh = the interpolation transposed applied to lx (at X of the step, in d.X)
void launch_cap_adj_spread(const LbmParams& p, const DevState& d, const AdjCap& a, cudaStream_t st);
// after the fluid's backward step: lambda_F, the stencil and membrane terms of lx, the parameter sums, and the
// clearing of the step's fields (d holds the membrane forces and spread force of the step); four kernels
void launch_cap_adj_vertices(const LbmParams& p, const DevState& d, const AdjCap& a, cudaStream_t st);

// dL/drho0^c(x) of an initial equilibrium lattice S0 (f_i = f_eq,i(rho0, u0), linear in rho0 at fixed u0):
// sum_i lambda0^c[i][x - c_i] S0^c[i][x - c_i] / rho0^c(x), into drho (2 N floats).
void launch_adj_initial(const LbmParams& p, const float* S0, const float* lam0, float* drho, cudaStream_t st);

}  // namespace scbb
