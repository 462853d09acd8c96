// Internal declarations shared by the CUDA translation units of libscbb (sm_103a).
//
// Population storage: two lattices S[c][i][N] (structure of arrays, x fastest) of FP32, IEEE FP16 or BF16
// values; all arithmetic is FP32 in every case.  A lattice holds the post-collision populations of the
// last step, not yet streamed; streaming is a pull, f_i(x) = S[i][x - c_i].
// Links that end on a wall node (Eq. 11) store the bounced value in the slot the receiving node pulls from,
// so every pull is the same plain gather and the density of any node can be recomputed from S.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

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

// Spread force of the immersed boundary: 64-bit fixed point in units of 2^-40.  The spreading sums the vertices'
// contributions with integer atomics, which are associative, so the sums (and the step) are the same bits in
// whatever order the atomics land; |values| < 2^23.
// (Both conversions stay in FP32: scaling by a power of two is exact, and the integer <-> float conversions
// round once.)
typedef unsigned long long IbmF;
__device__ __forceinline__ IbmF ibm_fix(float v) { return (IbmF)__float2ll_rn(v * 0x1p40f); }
__device__ __forceinline__ float ibm_unfix(IbmF v) { return __ll2float_rn((long long)v) * 0x1p-40f; }

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
    int store;              // population storage: 0 FP32, 1 FP16 (__half), 2 BF16 (__nv_bfloat16), 3 / 4 FP16 /
                            // BF16 deviations from w_i rref^c (DevH, DevB); the S pointers point to that type
    float rref[2];          // reference densities of the deviation storages (0 otherwise)
    int b4cfg;              // shape of the row-vectorised bulk kernel, 0 .. B4_CONFIGS - 1 (scbb_autotune)
    int onsite;             // 1: resting walls (ulo = uhi = 0) and on-site velocity planes z = 1 (vlo), nz-2 (vhi)
    float vlo[3], vhi[3];
    long long wait_limit;   // polls of a bounded wait on asynchronous copies before it gives up (error bit 4)
};

// Shapes of the row-vectorised bulk kernel: (threads per CTA, CTAs per SM, fewest planes per z-segment) =
// 0: (512, 1, 6), 1: (256, 2, 6), 2: (512, 1, 3), 3: (256, 2, 3).
constexpr int B4_CONFIGS = 4;

// Deviation storages: a population f_i^c is stored as the 16-bit value of f_i^c - w_i rref^c.  The reference
// adds nothing to the moments that the kernels cannot fold in (sum_i w_i = 1, sum_i w_i c_i = 0), and a
// population near w_i rref^c keeps the 16-bit type's relative precision on its (small) deviation.  Every load
// adds the reference back and every store takes it off; the rounding of the mass-closing rest population
// works on the deviations: d_0 = (rho - rref) - sum_{i >= 1} d_i.
struct DevH {
    __half h;
};
struct DevB {
    __nv_bfloat16 h;
};
template <typename T>
struct is_dev {
    static constexpr bool value = false;
};
template <>
struct is_dev<DevH> {
    static constexpr bool value = true;
};
template <>
struct is_dev<DevB> {
    static constexpr bool value = true;
};
// the reference density of component c for storage type T (0 for the plain storages, at compile time)
template <typename T>
__device__ __forceinline__ float dev_ref(const LbmParams& p, int c) {
    if constexpr (is_dev<T>::value) return p.rref[c];
    else return 0.f;
}

// Calls f with a null pointer of the population storage type of `store` (float, __half, __nv_bfloat16, DevH or
// DevB), so a launcher instantiates the kernel for that type: with_storage(p.store, [&](auto* tag) { ... }).
template <class F>
inline void with_storage(int store, F&& f) {
    if (store == 1) f(static_cast<__half*>(nullptr));
    else if (store == 2) f(static_cast<__nv_bfloat16*>(nullptr));
    else if (store == 3) f(static_cast<DevH*>(nullptr));
    else if (store == 4) f(static_cast<DevB*>(nullptr));
    else f(static_cast<float*>(nullptr));
}
// The same for kernels that have no deviation form (the fused bulk kernels and their wall pass, which a context
// with a deviation storage never runs: it requires the two-kernel bulk phase); the deviation codes map to the
// plain 16-bit types so that the launchers compile.
template <class F>
inline void with_plain_storage(int store, F&& f) {
    if (store == 1 || store == 3) f(static_cast<__half*>(nullptr));
    else if (store == 2 || store == 4) f(static_cast<__nv_bfloat16*>(nullptr));
    else f(static_cast<float*>(nullptr));
}

// Population element access for each storage (values convert to and from FP32 at the load and store;
// FP16 and BF16 stores round to nearest even).  A four-node vector is 16 bytes in FP32 and 8 bytes in FP16
// or BF16.
__device__ __forceinline__ float pld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float pld(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float pld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
// the value a store of this storage type keeps (identity for FP32): collisions sum the stored values of the
// moving populations, so the rest population absorbs their rounding and the node's mass is exact up to
// one rounding
__device__ __forceinline__ float pround(float v, const float*) { return v; }
__device__ __forceinline__ float pround(float v, const __half*) { return __half2float(__float2half_rn(v)); }
__device__ __forceinline__ float pround(float v, const __nv_bfloat16*) {
    return __bfloat162float(__float2bfloat16_rn(v));
}
// Unbiased rounding of v to the storage type: the neighbour below or above, the one above with probability
// (v - below) / (above - below), for a uniform 16-bit draw u.  The rest population closes each node's mass;
// rounded to nearest it would carry the same error at every node of a uniform phase, step after step, and
// the total mass would drift.
__device__ __forceinline__ float pdither(float v, uint32_t, const float*) { return v; }
__device__ __forceinline__ float pdither(float v, uint32_t u, const __half*) {
    const float lo = __half2float(__float2half_rd(v)), hi = __half2float(__float2half_ru(v));
    return (hi - lo) * ((float)u * (1.f / 65536.f)) < v - lo ? hi : lo;
}
__device__ __forceinline__ float pdither(float v, uint32_t u, const __nv_bfloat16*) {
    const float lo = __bfloat162float(__float2bfloat16_rd(v)), hi = __bfloat162float(__float2bfloat16_ru(v));
    return (hi - lo) * ((float)u * (1.f / 65536.f)) < v - lo ? hi : lo;
}
// Two 16-bit draws (high and low half) for node n: the node index and the bits of its two densities, so that
// the draws change with the state from step to step, through the 32-bit finalizer of MurmurHash3.
__device__ __forceinline__ uint32_t dither_bits(unsigned int n, float ra, float rb) {
    uint32_t h = n * 0x9e3779b9u ^ __float_as_uint(ra) ^ (__float_as_uint(rb) << 7);
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
// coherent loads, for populations a kernel also writes (the pld loads go through the read-only path)
__device__ __forceinline__ float pldc(const float* p) { return *p; }
__device__ __forceinline__ float pldc(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float pldc(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void pst(float* p, float v) { *p = v; }
__device__ __forceinline__ void pst(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void pst(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ float4 pld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 pld4(const __half* p) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    __half2 a, b;
    memcpy(&a, &u.x, 4);
    memcpy(&b, &u.y, 4);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ float4 pld4(const __nv_bfloat16* p) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    __nv_bfloat162 a, b;
    memcpy(&a, &u.x, 4);
    memcpy(&b, &u.y, 4);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ void pst4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void pst4(__half* p, float4 v) {
    const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 u;
    memcpy(&u.x, &a, 4);
    memcpy(&u.y, &b, 4);
    *reinterpret_cast<uint2*>(p) = u;
}
__device__ __forceinline__ void pst4(__nv_bfloat16* p, float4 v) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    memcpy(&u.x, &a, 4);
    memcpy(&u.y, &b, 4);
    *reinterpret_cast<uint2*>(p) = u;
}
// The deviation storages hold their deviations in the plain 16-bit types: the same access functions.
__device__ __forceinline__ const __half* raw16(const DevH* p) { return reinterpret_cast<const __half*>(p); }
__device__ __forceinline__ __half* raw16(DevH* p) { return reinterpret_cast<__half*>(p); }
__device__ __forceinline__ const __nv_bfloat16* raw16(const DevB* p) { return reinterpret_cast<const __nv_bfloat16*>(p); }
__device__ __forceinline__ __nv_bfloat16* raw16(DevB* p) { return reinterpret_cast<__nv_bfloat16*>(p); }
__device__ __forceinline__ float pld(const DevH* p) { return pld(raw16(p)); }
__device__ __forceinline__ float pld(const DevB* p) { return pld(raw16(p)); }
__device__ __forceinline__ float pldc(const DevH* p) { return pldc(raw16(p)); }
__device__ __forceinline__ float pldc(const DevB* p) { return pldc(raw16(p)); }
__device__ __forceinline__ float pround(float v, const DevH* p) { return pround(v, raw16(p)); }
__device__ __forceinline__ float pround(float v, const DevB* p) { return pround(v, raw16(p)); }
__device__ __forceinline__ float pdither(float v, uint32_t u, const DevH* p) { return pdither(v, u, raw16(p)); }
__device__ __forceinline__ float pdither(float v, uint32_t u, const DevB* p) { return pdither(v, u, raw16(p)); }
__device__ __forceinline__ void pst(DevH* p, float v) { pst(raw16(p), v); }
__device__ __forceinline__ void pst(DevB* p, float v) { pst(raw16(p), v); }
__device__ __forceinline__ float4 pld4(const DevH* p) { return pld4(raw16(p)); }
__device__ __forceinline__ float4 pld4(const DevB* p) { return pld4(raw16(p)); }
__device__ __forceinline__ void pst4(DevH* p, float4 v) { pst4(raw16(p), v); }
__device__ __forceinline__ void pst4(DevB* p, float4 v) { pst4(raw16(p), v); }

// One capsule's constants on the device.
struct CapDev {
    float kS, C, kB, kV, mass, colour;
    double V0;
    int v0, nv, t0, nt;
};

// Device-side buffers of a context (all carved from the caller's workspace).
constexpr int BB_CAND_PER_TRI = 16;   // capacity of the element search's candidate list, per triangle
constexpr int PP_NBR = 16;     // neighbour capsules listed per capsule for the repulsion

struct DevState {
    float* S[2];            // populations, 2 * 19 * N values each, of the type LbmParams::store names; one
                            // lattice (S[1] == S[0]) when the two-kernel bulk phase updates it in place
    double* stage;          // with one lattice: host-I/O staging, 5 N doubles; else null (the spare lattice serves)
    float* rho;             // [2][N] densities of the last collision
    float* J;               // [3][N] momentum of the last stream (two-kernel bulk phase)
    float* u;               // [3][N] velocity incl. half force, written where the IBM mask is set
    IbmF* Fibm;             // [3][N] immersed boundary: spread force, fixed-point sums (ibm_fix)
    uint32_t* mask;         // [ceil(N/32)] IBM stencil bits
    float* wall_rho;        // [2 walls][2 comp][nxy] densities of the planes next to the walls
    float* ghost;           // [2 walls][2 comp][nxy] virtual densities of the wall planes
    double* red;            // reduction scratch
    int* err;               // [4] sticky device error word (bits: 1 Mach guard or non-positive density, 2 boundary
                            //     list out of step, 4 a bounded wait gave up); [2..3] the grid barrier of a batch
                            //     whose first context this is
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
    float* tcol;            // [NT] colour of each element (its capsule's, or the mesh's per-element colour)
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
    // ---- bounce-back coupling (coupling == 0)
    uint16_t* owner;        // [N] 0 outside every capsule, k+1 inside capsule k, 0xFFFF wall node
    uint32_t* bmask;        // [ceil(N/32)] boundary-node bits (nodes with a cut membrane link)
    uint32_t* fmask;        // [ceil(N/32)] fresh-node bits of the current step
    int* blist;             // [maxB] boundary nodes
    float2* bdm;            // [maxB] mass change (A, B) of the bounce-back links, one partial per block of the
                            //     boundary kernel (cnt[5] partials)
    int* belem;             // [maxB][18] element crossed by the link along direction i (slot i-1), -1 if uncut
    unsigned long long* bkey;   // [maxB][18] nearest crossing found so far: (parameter bits << 32) | triangle
    int4* lcand;            // [NT * BB_CAND_PER_TRI] crossing candidates of the element search: (t, X, Y, Z << 5 | i)
    int* bidx;              // [N] place in the boundary list of each node listed by the last list build (-1: the
                            //     list was full); stale for the other nodes
    int* flist;             // [maxF] fresh nodes
    int* fold;              // [maxF] their owner before the change
    float4* fnew;           // [maxF][2] new (rhoA, rhoB, ok, -) and (vx, vy, vz, element)
    int* cnt;               // [8] 0: boundary nodes, 1: fresh nodes, 2: overflow flags, 4: fresh nodes of the
                            //     previous step (saved before re-listing), 5: partials in bdm, 6: cut links
                            //     whose element came from the nearest-centroid rule (running count),
                            //     7: crossing candidates of the element search
    float4* emom;           // [2][NT] exchanged momentum (Eq. 12) by step parity
    float4* epend;          // [2][NT] Shan-Chen reactions and fresh-node momenta by step parity
    int4* cbox;             // [NM][2] classification box (lo, hi), unwrapped lattice coordinates
    int* ccnt;              // [NM][CW*CW] crossings per column
    float* czs;             // [NM][CW*CW][MAXC] crossing heights
    float2* fdm;            // [maxF] mass change (A, B) of each fresh node's replacement
    float4* trec;           // [NT][4] vertex positions and centroid of every triangle at X(t+1); the centroid's w
                            //     holds the triangle's capsule (int bits)
    int* tcnt;              // [NM][CW*CW] triangles whose xy bounding box overlaps each column cell
    int4* tlst;             // [NM][CW*CW][BB_MAXT] their ids and z ranges (t, zmin bits, zmax bits, 0)
    float4* vrho;           // [N] at boundary nodes: mean rho^A, rho^B over neighbours on the other side,
                            //     count, 1 if those neighbours lie on more than one other side
    double* mass;           // [8] 0-1: M(0), 2-3: mass change since M(0) (FP64 running sums of the bounce-back and
                            //     fresh-node changes), 4-5: correction factors
    int maxB, maxF, CW;
    // particle-particle repulsion (several capsules)
    int* pp_head;           // [pp_size] hashed cell heads, nullptr when unused
    int* pp_next;           // [NV] linked lists
    float4* Fpp;            // [NV] repulsion force of the step
    float4* pp_ref;         // [NM] reference point of each capsule for the step's repulsion (its centre)
    int* pp_rmax;           // [NM] largest distance of the capsule's vertices from pp_ref (float bits)
    int* pp_nbr;            // [NM][PP_NBR] capsules whose bounding spheres come within the repulsion range
    int* pp_ncnt;           // [NM] their number, -1 when more than PP_NBR
    int pp_size;
    float pp_eps, pp_d0;
    double rho_maj, rho_min, C0;
    int mass_correction;
};

constexpr int BB_MAXC = 16;             // crossings stored per classification column
constexpr int BB_MAXT = 96;             // triangles listed per column cell
constexpr float BB_EPSX = 1.37e-4f;     // offsets of the classification rays / link segments
constexpr float BB_EPSY = 2.91e-4f;
constexpr float BB_EPSZ = 3.53e-4f;

// ---- device helpers shared by the kernels ----
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
// Pull helper: populations arriving at (gx, gy, z) from its 18 neighbours (x, y periodic).
// ------------------------------------------------------------------------------------------------------
struct Cols {
    int cx[3];          // x - 1, x, x + 1 (wrapped)
    int ry[3];          // (y - 1) nx, y nx, (y + 1) nx (wrapped)
};

template <typename T>
__device__ __forceinline__ void pull(const LbmParams& p, const T* __restrict__ S, const Cols& k, int z,
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
        f[i] = pld(S + (size_t)i * p.N + m);
        f[Q + i] = pld(S + (size_t)(Q + i) * p.N + m);
        if constexpr (is_dev<T>::value) {
            f[i] += dir_w(i) * p.rref[0];
            f[Q + i] += dir_w(i) * p.rref[1];
        }
    }
}

// On-site velocity boundary (Zou and He, in the D3Q19 form of Hecht and Harting; Sec. III.A and III.C impose the
// shear with it).  f: the 2 x 19 populations pulled at a node of plane z = 1 (velocity vlo) or z = nz-2 (vhi),
// the ones that arrived from the wall included.  Those are replaced, component by component, so that the
// node's velocity is the plane's velocity U: with n the inward normal, rho = (sum of the populations with
// c.n = 0 + 2 x those with c.n < 0) / (1 - U.n) and, for c_i.n > 0,
// f_i = f_opp(i) + 6 w_i rho c_i.U - c_i,t . N_t with N_t = 1/2 sum_{c.n = 0} f c_t - rho U_t / 3.
__device__ __forceinline__ bool is_onsite_plane(const LbmParams& p, int z) {
    return p.onsite && (z == 1 || z == p.nz - 2);
}
__device__ __forceinline__ void onsite_fix(const LbmParams& p, int z, float (&f)[2 * Q]) {
    const int nrm = z == 1 ? 1 : -1;
    const float* U = nrm > 0 ? p.vlo : p.vhi;
#pragma unroll
    for (int c = 0; c < 2; c++) {
        float s0 = 0.f, sin = 0.f, tx = 0.f, ty = 0.f;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const float v = f[c * Q + i];
            if (dir_z(i) == 0) {
                s0 += v;
                if (dir_x(i)) tx += dir_x(i) * v;
                if (dir_y(i)) ty += dir_y(i) * v;
            } else if (dir_z(i) == -nrm) {
                sin += v;
            }
        }
        const float rho = (s0 + 2.f * sin) / (1.f - nrm * U[2]);
        const float Nx = 0.5f * tx - rho * U[0] * (1.f / 3.f), Ny = 0.5f * ty - rho * U[1] * (1.f / 3.f);
#pragma unroll
        for (int i = 1; i < Q; i++)
            if (dir_z(i) == nrm)
                f[c * Q + i] = f[c * Q + dir_opp(i)] +
                               6.f * dir_w(i) * rho * (dir_x(i) * U[0] + dir_y(i) * U[1] + dir_z(i) * U[2]) -
                               (dir_x(i) * Nx + dir_y(i) * Ny);
    }
}

// ---- launches (lbm_kernels.cu) ----
void launch_init_state(const LbmParams& p, float* S, const float* rho_st, const float* u_st, cudaStream_t st);
void launch_init_state(const LbmParams& p, float* S, const double* rho_st, const double* u_st, cudaStream_t st);
void launch_wall_ghost(const LbmParams& p, const float* S, float* wall_rho, float* ghost, cudaStream_t st);
// mode 0: fluid only (also with bounce-back membranes), 1: immersed boundary (mask = IBM stencil bits)
// J: [3][N] momentum scratch of the two-kernel bulk phase (tau = 1), which also writes the wall ghost
// densities itself (bulk_writes_ghost); with J null the fused kernels run
void launch_bulk(const LbmParams& p, const float* S, float* D, float* rho, float* J, float* ghost,
                 const IbmF* Fibm, const uint32_t* mask, float* u, int* err, int mode, cudaStream_t st);
// true when the bounce-back coupling can run on this lattice: the two-kernel bulk phase or the fused
// row-vectorised kernel (both store every node of the lattice whole)
bool bulk_vectorised(const LbmParams& p);
bool bulk_writes_ghost(const LbmParams& p);
int bulk_variant();

// ---- the two-kernel bulk phase (bulk_split.cu)
bool bulk_split(const LbmParams& p);
int split_grid_blocks(const LbmParams& p);
void launch_split(const LbmParams& p, const float* S, float* D, float* rho, float* J, float* ghost,
                  const IbmF* Fibm, const uint32_t* mask, float* u, int* err, int mode, cudaStream_t st);

// Bulk phase of a batch of boxes in one cooperative launch (kernel parameters carry every box).
constexpr int BATCH_MAX = 64;
constexpr int BATCH_THREADS = 256;
struct BatchBox {
    LbmParams p;
    const void* S;          // populations read (storage type of p.store)
    void* D;                // populations written
    float* rho;
    float* J;
    float* ghost;
    const IbmF* Fibm;
    const uint32_t* mask;
    float* u;
    int* err;
    unsigned int a_begin;   // first thread of kernel A (a multiple of 32)
    unsigned int a_count;   // its work units: quads (vec) or nodes
    int b_begin;            // first (tile, z-segment) item of kernel B
    int cols, nseg, TY, vec;
};
struct BatchDesc {
    int nbox;
    unsigned int a_total;
    int b_total;
    int* bar;               // [2] grid barrier: arrivals, generation
    long long spin_limit;   // polls of a barrier wait before it gives up
    BatchBox box[BATCH_MAX];
};
bool launch_batch_bulk(BatchDesc& d, int mode, int store, cudaStream_t st);
// what: 0 fields (rho^A, rho^B, u: 5 N floats), 1 populations [c][n][i], 2 / 3 one component's [n][i],
// 4 fields in FP64 into out64 (5 N doubles), 16 + c Q + i one direction of one component (N floats)
void launch_export(const LbmParams& p, const float* S, float* out, int what, cudaStream_t st, double* out64 = nullptr);
void launch_moments_reduce(const LbmParams& p, const float* S, double* red, cudaStream_t st);
int bulk_grid_blocks(const LbmParams& p);

// ---- launches (membrane_kernels.cu) ----
void launch_capsule_reduce(const DevState& d, cudaStream_t st);
// returns the number of kernels launched
int launch_membrane_forces(const LbmParams& p, const DevState& d, bool bb, int step, cudaStream_t st);
int launch_ibm_spread(const LbmParams& p, const DevState& d, cudaStream_t st);
void launch_ibm_interp(const LbmParams& p, const DevState& d, cudaStream_t st);
int launch_pp_forces(const LbmParams& p, const DevState& d, float eps, float d0, cudaStream_t st);

// ---- launches (bb_kernels.cu) ----
void launch_bb_init(const LbmParams& p, const DevState& d, cudaStream_t st);
void launch_bb_classify(const LbmParams& p, const DevState& d, int step, bool init, cudaStream_t st);
void launch_bb_boundary(const LbmParams& p, const DevState& d, const float* S, float* D, const float* ghost,
                        int step, int* err, cudaStream_t st);
void launch_bb_fresh(const LbmParams& p, const DevState& d, float* Snew, int step,
                     cudaStream_t st);

}  // namespace scbb
