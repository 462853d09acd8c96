// Half-way bounce-back coupling of membranes and fluid (Sec. II.C-II.E), sm_103a.
//
//   classification   owner field from z-ray parity per lattice column, updated in place inside each
//                    capsule's box; nodes that change side are recorded as fresh
//   boundary list    nodes with a cut membrane link; for each cut link the crossed triangle
//   boundary kernel  collision of the boundary nodes with Shan-Chen virtual densities and the wetting offset
//                    (Eq. 14-15), moving half-way bounce-back (Eq. 11) and the exchanged momentum (Eq. 12)
//   fresh nodes      new density from the non-fresh neighbours on the new side (Eq. 16), adaptive mass
//                    correction (Eq. 18), velocity of the nearest element (Eq. 17), momentum balance
//
// Geometry readings shared with the FP64 oracle: a node is inside capsule k when the +z ray from
// (x + EPSX, y + EPSY, z + EPSZ) crosses its surface an odd number of times (a crossing counts when the
// offset point lies strictly inside the triangle's xy projection and the triangle is above it); a link is
// cut when its two nodes have different owners, and its element is the triangle the offset segment
// crosses, the crossing nearest to the node of lower linear index (no crossing: nearest centroid to the
// link midpoint).
#include <cuda_fp16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include "bb.cuh"
#include "pdl.cuh"
#include "scbb_internal.cuh"

namespace scbb {

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ bool wall_z(const LbmParams& p, int z) { return p.walls && (z == 0 || z == p.nz - 1); }

// a wrapped into 0 .. n-1; coordinates already in range (almost all) skip the integer modulo
__device__ __forceinline__ int wrapf(int a, int n) { return (unsigned)a < (unsigned)n ? a : wrapi(a, n); }

// linear index of unwrapped lattice coordinates (x, y periodic; z periodic without walls), -1 outside
__device__ __forceinline__ long long node_of(const LbmParams& p, int x, int y, int z) {
    x = wrapf(x, p.nx);
    y = wrapf(y, p.ny);
    if (p.walls) {
        if (z < 0 || z >= p.nz) return -1;
    } else {
        z = wrapf(z, p.nz);
    }
    return (long long)x + (long long)p.nx * (y + (long long)p.ny * z);
}

// Grid-stride launches over the boundary and fresh lists: the lists' lengths live on the device, so the
// grid fills every SM at the kernel's occupancy (at most the blocks the list capacity needs) and each warp
// or thread strides over the entries.
static int sm_count() {
    static const int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
            v = 152;
        return v;
    }();
    return n;
}
static int occupancy(const void* kernel, int threads) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, 0) != cudaSuccess || v < 1) v = 1;
    return v;
}
// Blocks of 128 threads per capsule for a pass over each capsule's box of `nodes` nodes: about 16 blocks per SM
// in all, at most one per 128 nodes.
static unsigned box_blocks(const DevState& d, size_t nodes) {
    const size_t per_cap = ((size_t)16 * sm_count() + d.NM - 1) / (d.NM > 0 ? d.NM : 1);
    const size_t full = (nodes + 127) / 128;
    const size_t g = per_cap < full ? per_cap : full;
    return (unsigned)(g > 0 ? g : 1);
}

static unsigned fill_grid(int per_sm, size_t need) {
    size_t g = (size_t)per_sm * sm_count();
    if (need < g) g = need;
    return (unsigned)(g > 0 ? g : 1);
}

// coordinate of lattice index q in the periodic image nearest to r (period L; per = periodic)
__device__ __forceinline__ float near_image(int q, float r, int L, bool per) {
    float v = (float)q;
    if (per) v -= L * floorf((v - r) / L + 0.5f);
    return v;
}

// A bounding-box interval [lo, hi] in one int as the FP16 pair (lo rounded down, -hi rounded up in
// magnitude), so the packed box always contains the exact one: a filter on it keeps every triangle the exact
// box keeps.  A query interval [q0, q1] is packed as (q1 rounded up, -q0 with q0 rounded down); the two
// intervals meet exactly when lo <= q1 and -hi <= -q0, one paired FP16 comparison.
__device__ __forceinline__ int pack_range(float lo, float hi) {
    const unsigned a = __half_as_ushort(__float2half_rd(lo));
    const unsigned b = __half_as_ushort(__hneg(__float2half_ru(hi)));
    return (int)(a | (b << 16));
}
__device__ __forceinline__ __half2 as_half2(int v) {
    return __halves2half2(__ushort_as_half((unsigned short)(v & 0xffff)),
                          __ushort_as_half((unsigned short)((unsigned)v >> 16)));
}
__device__ __forceinline__ __half2 query_range(float q0, float q1) {
    return __halves2half2(__float2half_ru(q1), __hneg(__float2half_rd(q0)));
}
struct QueryBox {
    __half2 z, x, y;
};
__device__ __forceinline__ QueryBox query_box(float3 q0, float3 q1) {
    QueryBox b;
    b.z = query_range(q0.z, q1.z);
    b.x = query_range(q0.x, q1.x);
    b.y = query_range(q0.y, q1.y);
    return b;
}
// list entry (t, z range, x range, y range) against the query box
__device__ __forceinline__ bool entry_meets(int4 e, const QueryBox& b) {
    return __hble2(as_half2(e.y), b.z) && __hble2(as_half2(e.z), b.x) && __hble2(as_half2(e.w), b.y);
}

// The triangle lists of a w x w block of column cells of one capsule, read by a warp as one flat list:
// lane j (j < w*w) holds cell j's column and the inclusive end of its entries, so that every lane loads
// its count in parallel and the warp then strides over all entries together.
struct CellScan {
    int col;      // column index of this lane's cell, -1 outside the capsule's cell grid
    int end;      // inclusive prefix sum of the entry counts up to this lane's cell
    int total;    // entries of all w*w cells
};

__device__ __forceinline__ CellScan cell_scan(const DevState& d, int cap, int cx0, int cy0, int w, int lane) {
    CellScan s;
    s.col = -1;
    int c = 0;
    if (lane < w * w) {
        const int cx = cx0 + lane % w, cy = cy0 + lane / w;
        if (cx >= 0 && cy >= 0 && cx < d.CW && cy < d.CW) {
            s.col = cap * d.CW * d.CW + cy * d.CW + cx;
            c = min(d.tcnt[s.col], BB_MAXT);
        }
    }
    s.end = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, s.end, o);
        if (lane >= o) s.end += v;
    }
    s.total = __shfl_sync(0xffffffffu, s.end, 31);
    return s;
}

// Position in the triangle list of entry k < total of the flat list (warp-convergent call; any k).
__device__ __forceinline__ size_t cell_entry(const CellScan& s, int k) {
    int j = 0;                    // cell of entry k: the number of cells whose entries end at or before k
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        if (__shfl_sync(0xffffffffu, s.end, j + o - 1) <= k) j += o;
    // every lane takes part in the shuffles with its own j; a cell outside the grid holds no entries, so
    // only k >= total can land on one
    const int col = __shfl_sync(0xffffffffu, s.col, j);
    const int prev = __shfl_sync(0xffffffffu, s.end, j > 0 ? j - 1 : 0);
    const int start = j > 0 ? prev : 0;
    return col < 0 ? 0 : (size_t)col * BB_MAXT + (size_t)(k - start);
}

// Streams the entries of a CellScan whose boxes meet the query box [q0, q1] through a per-warp queue of
// CAND_Q ids in shared memory, so that the per-candidate work runs on full warps: fn(t) is called by the
// whole warp, each lane with a candidate triangle t or with -1.  Two entries per lane are loaded per round
// (independent loads in flight).  A triangle listed in several cells may come more than once.
constexpr int CAND_Q = 96;

template <class Fn>
__device__ __forceinline__ void for_candidates(const DevState& d, const CellScan& cs, float3 q0, float3 q1,
                                               int* queue, int lane, Fn&& fn) {
    const QueryBox qb = query_box(q0, q1);
    int qn = 0;                                   // warp-uniform queue length
    auto enqueue = [&](bool keep, int t) {
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) queue[qn + __popc(bal & ((1u << lane) - 1u))] = t;
        qn += __popc(bal);
    };
    for (int base = 0; base < cs.total; base += 64) {
        const int k0 = base + lane, k1 = base + 32 + lane;
        const size_t a0 = cell_entry(cs, k0), a1 = cell_entry(cs, k1);
        int4 e0 = make_int4(-1, 0, 0, 0), e1 = make_int4(-1, 0, 0, 0);
        if (k0 < cs.total) e0 = d.tlst[a0];
        if (k1 < cs.total) e1 = d.tlst[a1];
        enqueue(k0 < cs.total && entry_meets(e0, qb), e0.x);
        enqueue(k1 < cs.total && entry_meets(e1, qb), e1.x);
        __syncwarp();
        while (qn >= 32) {
            const int tt = queue[lane];
            __syncwarp();
            if (lane < qn - 32) queue[lane] = queue[32 + lane];
            if (lane + 32 < qn - 32) queue[lane + 32] = queue[64 + lane];
            __syncwarp();
            qn -= 32;
            fn(tt);
            __syncwarp();
        }
    }
    if (qn > 0) {
        const int tt = lane < qn ? queue[lane] : -1;
        __syncwarp();
        fn(tt);
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------------------
// Classification
// ------------------------------------------------------------------------------------------------------

// Per triangle: clear the element accumulators the next step will fill, and append the heights where the
// triangle crosses the +z rays of the columns inside its xy projection.
__global__ void k_class_tri(LbmParams p, DevState d, int step) {
    pdl_wait();
    pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) { d.cnt[0] = 0; d.cnt[1] = 0; d.cnt[7] = 0; }
    if (t >= d.NT) return;
    const int nxt = (step + 1) & 1;
    d.emom[nxt * d.NT + t] = make_float4(0.f, 0.f, 0.f, 0.f);
    d.epend[nxt * d.NT + t] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int4 T = d.tri[t];
    const int k = T.w;
    const int4 lo = d.cbox[2 * k];
    const float3 a = f3(d.X[T.x]), b = f3(d.X[T.y]), c = f3(d.X[T.z]);
    // compact record for the element searches of this step
    d.trec[4 * t + 0] = make_float4(a.x, a.y, a.z, 0.f);
    d.trec[4 * t + 1] = make_float4(b.x, b.y, b.z, 0.f);
    d.trec[4 * t + 2] = make_float4(c.x, c.y, c.z, 0.f);
    d.trec[4 * t + 3] = make_float4((a.x + b.x + c.x) * (1.f / 3.f), (a.y + b.y + c.y) * (1.f / 3.f),
                                    (a.z + b.z + c.z) * (1.f / 3.f), __int_as_float(k));
    const float xmin = fminf(a.x, fminf(b.x, c.x)), xmax = fmaxf(a.x, fmaxf(b.x, c.x));
    const float ymin = fminf(a.y, fminf(b.y, c.y)), ymax = fmaxf(a.y, fmaxf(b.y, c.y));
    // a triangle wider than a column grid or outside its capsule's grid (a degenerate mesh, runaway or
    // non-finite vertices) is flagged and skipped, so that the loops below visit at most CW + 3 columns of
    // bounded coordinates
    if (!(xmax - xmin < (float)d.CW && ymax - ymin < (float)d.CW && xmin >= (float)(lo.x - 2) &&
          xmax <= (float)(lo.x + d.CW + 2) && ymin >= (float)(lo.y - 2) && ymax <= (float)(lo.y + d.CW + 2))) {
        atomicOr(d.cnt + 2, 32);
        return;
    }
    // column cells [xx, xx+1) x [yy, yy+1) overlapped by the xy bounding box: candidate lists for the
    // element searches
    for (int yy = (int)floorf(ymin); yy <= (int)floorf(ymax); yy++)
        for (int xx = (int)floorf(xmin); xx <= (int)floorf(xmax); xx++) {
            const int cx = xx - lo.x, cy = yy - lo.y;
            if (cx < 0 || cy < 0 || cx >= d.CW || cy >= d.CW) { atomicOr(d.cnt + 2, 1); continue; }
            const int col = k * d.CW * d.CW + cy * d.CW + cx;
            const int slot = atomicAdd(d.tcnt + col, 1);
            if (slot < BB_MAXT)
                d.tlst[(size_t)col * BB_MAXT + slot] =
                    make_int4(t, pack_range(fminf(a.z, fminf(b.z, c.z)), fmaxf(a.z, fmaxf(b.z, c.z))),
                              pack_range(xmin, xmax), pack_range(ymin, ymax));
            else atomicOr(d.cnt + 2, 64);
        }
    const float det = (b.x - a.x) * (c.y - a.y) - (c.x - a.x) * (b.y - a.y);
    if (det == 0.f) return;
    const int x0 = (int)ceilf(xmin - BB_EPSX), x1 = (int)floorf(xmax - BB_EPSX);
    const int y0 = (int)ceilf(ymin - BB_EPSY), y1 = (int)floorf(ymax - BB_EPSY);
    for (int yy = y0; yy <= y1; yy++)
        for (int xx = x0; xx <= x1; xx++) {
            const float px = xx + BB_EPSX - a.x, py = yy + BB_EPSY - a.y;
            const float l1 = (px * (c.y - a.y) - (c.x - a.x) * py) / det;
            const float l2 = ((b.x - a.x) * py - px * (b.y - a.y)) / det;
            const float l0 = 1.f - l1 - l2;
            if (l0 <= 0.f || l1 <= 0.f || l2 <= 0.f) continue;
            const int cx = xx - lo.x, cy = yy - lo.y;
            if (cx < 0 || cy < 0 || cx >= d.CW || cy >= d.CW) { atomicOr(d.cnt + 2, 1); continue; }
            const int col = k * d.CW * d.CW + cy * d.CW + cx;
            const int slot = atomicAdd(d.ccnt + col, 1);
            if (slot < BB_MAXC) d.czs[(size_t)col * BB_MAXC + slot] = l0 * a.z + l1 * b.z + l2 * c.z;
            else atomicOr(d.cnt + 2, 2);
        }
}

// One thread per node of a capsule's box: parity of the column's crossings above the node; owner updated in
// place, changed nodes recorded as fresh.
__device__ __forceinline__ void class_col_node(const LbmParams& p, const DevState& d, int init, int k, int4 lo,
                                               int4 hi, int q) {
    const int c = q % (d.CW * d.CW), zo = q / (d.CW * d.CW);
    if (zo >= d.CW) return;
    const int cx = c % d.CW, cy = c / d.CW;
    const int xx = lo.x + cx, yy = lo.y + cy, zz = lo.z + zo;
    if (xx > hi.x || yy > hi.y || zz > hi.z) return;
    if (p.walls && (zz < 1 || zz > p.nz - 2)) return;
    const long long n = node_of(p, xx, yy, zz);
    if (n < 0) return;
    const uint16_t old = d.owner[n];
    if (old == 0xFFFF) return;
    const int col = k * d.CW * d.CW + c;
    const int nc = min(d.ccnt[col], BB_MAXC);
    const float pz = zz + BB_EPSZ;
    int above = 0;
    for (int j = 0; j < nc; j++) above += d.czs[(size_t)col * BB_MAXC + j] > pz;
    const uint16_t me = (uint16_t)(k + 1);
    uint16_t nw = old;
    if (above & 1) nw = me;
    else if (old == me) nw = 0;
    if (nw == old) return;
    d.owner[n] = nw;
    if (init) return;
    const int f = atomicAdd(d.cnt + 1, 1);
    if (f < d.maxF) {
        d.flist[f] = (int)n;
        d.fold[f] = old;
        atomicOr(d.fmask + (n >> 5), 1u << (n & 31));
    } else {
        atomicOr(d.cnt + 2, 4);
    }
}

// Grid-stride over each capsule's box (blockIdx.y: the capsule): a few blocks per capsule rather than a block
// per 128 nodes, whose launch and drain cost more than their work with hundreds of capsules.
__global__ void k_class_col(LbmParams p, DevState d, int init) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.y;
    const int4 lo = d.cbox[2 * k], hi = d.cbox[2 * k + 1];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.CW * d.CW * d.CW; q += gridDim.x * blockDim.x)
        class_col_node(p, d, init, k, lo, hi, q);
}

// Clears the boundary and fresh bits of the previous step's lists (and the boundary nodes' places, so that
// bidx is -1 at every node not listed) and the per-column counters.
__global__ void k_lists_reset(DevState d) {
    pdl_wait();
    pdl_trigger();
    const int nb = d.cnt[0], nf = d.cnt[1];
    if (blockIdx.x == 0 && threadIdx.x == 0) d.cnt[4] = nf;     // fresh nodes replaced at the end of the previous step
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < d.NM * d.CW * d.CW; q += gridDim.x * blockDim.x) {
        d.ccnt[q] = 0;
        d.tcnt[q] = 0;
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < max(nb, nf); q += gridDim.x * blockDim.x) {
        if (q < nb && q < d.maxB) {
            const int n = d.blist[q];
            atomicAnd(d.bmask + (n >> 5), ~(1u << (n & 31)));
            d.bidx[n] = -1;
        }
        if (q < nf && q < d.maxF) {
            const int n = d.flist[q];
            atomicAnd(d.fmask + (n >> 5), ~(1u << (n & 31)));
        }
    }
}

// Nodes of each capsule's box (one node wider) with a cut membrane link join the boundary list; each one's
// place in it goes to bidx, and the crossing keys of its links start at "none".
__device__ __forceinline__ void mark_node(const LbmParams& p, const DevState& d, int k, int4 lo, int wx, int wy,
                                          int q) {
    const int xx = lo.x - 1 + q % wx, yy = lo.y - 1 + (q / wx) % wy, zz = lo.z - 1 + q / (wx * wy);
    // A node can have a link to capsule k's inside only if its column or a neighbouring one crosses capsule k's
    // surface (elsewhere no node is k's: the ray parity is even); links between other sides are listed by the
    // passes of the capsules whose insides they touch.
    const int ccx = xx - lo.x, ccy = yy - lo.y;
    bool crossed = false;
    for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
            const int cx = ccx + dx, cy = ccy + dy;
            if (cx >= 0 && cy >= 0 && cx < d.CW && cy < d.CW && d.ccnt[k * d.CW * d.CW + cy * d.CW + cx] > 0)
                crossed = true;
        }
    if (!crossed) return;
    const long long n = node_of(p, xx, yy, zz);
    if (n < 0) return;
    const uint16_t me = d.owner[n];
    if (me == 0xFFFF) return;
    bool cut = false;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const long long m = node_of(p, xx + dir_x(i), yy + dir_y(i), zz + dir_z(i));
        if (m < 0) continue;
        const uint16_t o = d.owner[m];
        if (o != 0xFFFF && o != me) cut = true;
    }
    if (!cut) return;
    const uint32_t bit = 1u << (n & 31);
    const uint32_t prev = atomicOr(d.bmask + (n >> 5), bit);
    if (prev & bit) return;                           // already listed (boxes of two capsules overlap)
    const int b = atomicAdd(d.cnt + 0, 1);
    d.bidx[n] = b < d.maxB ? b : -1;
    if (b < d.maxB) {
        d.blist[b] = (int)n;
        // no crossing yet on any of its links (the element search lowers these keys)
        ulonglong2* k2 = reinterpret_cast<ulonglong2*>(d.bkey + (size_t)b * (Q - 1));
#pragma unroll
        for (int j = 0; j < (Q - 1) / 2; j++) k2[j] = make_ulonglong2(~0ull, ~0ull);
    } else {
        atomicOr(d.cnt + 2, 8);
    }
}

// Grid-stride over each capsule's box, one node wider (blockIdx.y: the capsule).
__global__ void k_boundary_mark(LbmParams p, DevState d) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.y;
    const int4 lo = d.cbox[2 * k], hi = d.cbox[2 * k + 1];
    const int wx = hi.x - lo.x + 3, wy = hi.y - lo.y + 3, wz = hi.z - lo.z + 3;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < wx * wy * wz; q += gridDim.x * blockDim.x)
        mark_node(p, d, k, lo, wx, wy, q);
}

// ------------------------------------------------------------------------------------------------------
// Crossed elements of the cut links
// ------------------------------------------------------------------------------------------------------
// A cut link's element is the triangle its segment crosses nearest to the node of lower linear index (lower
// triangle id on ties).  The search runs over the triangles: a thread per triangle and group of link
// directions visits the lattice links whose segments can meet its bounding box and, for each cut link the
// triangle crosses, records the key
// (crossing parameter, triangle id) with a 64-bit atomicMin at every boundary node that searches this
// triangle's capsule along that link: the minimum over all triangles is the nearest crossing whatever the
// order.  Each node takes the link's segment as it would alone: from its own offset position in the periodic
// image nearest the capsule's centre, along c_i, turned around to start at the node of lower linear index.
// Links left without a crossing (round-off) are resolved when the list is read (k_bb_vrho).

// The segment's bounding box meets the triangle's [b0, b1].
__device__ __forceinline__ bool seg_meets_box(float3 P, float3 Dv, float3 b0, float3 b1) {
    if (fmaxf(P.x, P.x + Dv.x) < b0.x || fminf(P.x, P.x + Dv.x) > b1.x) return false;
    if (fmaxf(P.y, P.y + Dv.y) < b0.y || fminf(P.y, P.y + Dv.y) > b1.y) return false;
    if (fmaxf(P.z, P.z + Dv.z) < b0.z || fminf(P.z, P.z + Dv.z) > b1.z) return false;
    return true;
}

// Segment P + s Dv (s in [0, 1]) against the triangle (v0, v0 + e1, v0 + e2): Moller-Trumbore with closed
// bounds; the crossing parameter in tt (a crossing at s = -0 counts as +0, so the key orders it first).
__device__ __forceinline__ bool seg_tri(float3 P, float3 Dv, float3 v0, float3 e1, float3 e2, float& tt) {
    const float3 h = cross(Dv, e2);
    const float det = dot(e1, h);
    if (fabsf(det) < 1e-30f) return false;
    const float inv = 1.f / det;
    const float3 sv = sub(P, v0);
    const float u = dot(sv, h) * inv;
    if (u < 0.f || u > 1.f) return false;
    const float3 qv = cross(sv, e1);
    const float v = dot(Dv, qv) * inv;
    if (v < 0.f || u + v > 1.f) return false;
    tt = dot(e2, qv) * inv;
    if (tt < 0.f || tt > 1.f) return false;
    tt = __fadd_rn(tt, 0.f);
    return true;
}

struct TriGeom {
    float3 v0, e1, e2, b0, b1, cr;   // vertex 0, edges, bounding box, capsule centre (image reference)
    int t, k;
};

// Lattice coordinate X (unwrapped) is the periodic image of its node nearest the capsule's centre r, as
// near_image takes it: at once when X lies well inside half a period of r, else by near_image itself.
__device__ __forceinline__ bool own_image(int X, float r, int L, bool per) {
    if (!per || fabsf((float)X - r) < 0.5f * (float)L - 1.f) return true;
    return near_image(wrapf(X, L), r, L, true) == (float)X;
}

// The segment node n (unwrapped coordinates X, Y, Z, its own image) tests along direction i towards its
// neighbour o: from its offset position, turned around to start at the node of lower linear index.
__device__ __forceinline__ void end_segment(long long n, long long o, int X, int Y, int Z, int i, float3& P,
                                            float3& Dv) {
    P = make_float3((float)X + BB_EPSX, (float)Y + BB_EPSY, (float)Z + BB_EPSZ);
    Dv = make_float3((float)dir_x(i), (float)dir_y(i), (float)dir_z(i));
    if (o < n) {
        P = make_float3(P.x + Dv.x, P.y + Dv.y, P.z + Dv.z);
        Dv = make_float3(-Dv.x, -Dv.y, -Dv.z);
    }
}

// Crossing parameter of the triangle on a segment, -1 when it misses.
__device__ __forceinline__ float seg_cross(const TriGeom& g, float3 P, float3 Dv) {
    float tt;
    if (!seg_meets_box(P, Dv, g.b0, g.b1) || !seg_tri(P, Dv, g.v0, g.e1, g.e2, tt)) return -1.f;
    return tt;
}

// Records the crossing (parameter tt >= 0) at node n's link along direction i, when n is listed.
__device__ __forceinline__ void end_record(const DevState& d, const TriGeom& g, int b, int i, float tt) {
    if (b < 0) return;              // not listed: the list is full (flagged by the list kernel)
    const unsigned long long key = ((unsigned long long)__float_as_uint(tt) << 32) | (unsigned long long)(unsigned)g.t;
    atomicMin(d.bkey + (size_t)b * (Q - 1) + (i - 1), key);
}

// Crossing candidates, one thread per (triangle, group of the nine directions c_i with odd i): G = 3 groups of an
// axis and two face diagonals ({1,7,13} {3,9,15} {5,11,17}) for many triangles, G = 9 single directions for few
// (more threads, shorter ones).  The nine odd directions and their opposites (i + 1, the same links seen from
// the other end) are all eighteen.  A link whose segment can meet the triangle's box goes through two cheap
// conservative tests (its ends straddle the triangle's plane; where it meets the plane lies in the box) and,
// if it passes, onto the candidate list (t, X, Y, Z << 5 | i) that k_link_test takes a thread per entry: the
// enumeration's uneven loops and the few survivors would otherwise leave most lanes idle in the exact tests.
// The enumeration runs twice, to count and to write, so that a warp takes its places with one atomic.
constexpr int LC_CAP = BB_CAND_PER_TRI;     // candidate capacity per triangle (a few survive on average)

// The links of direction c_i (odd i) whose segment can meet the triangle's box (v0, e1, e2; box b0, b1) and that
// pass the two cheap tests: f(X, Y, Z) for each.
template <class F>
__device__ __forceinline__ void link_candidates(int i, float3 v0, float3 b0, float3 b1, float3 nrm, float tol, F&& f) {
    constexpr float DL = 1e-3f;     // margin of the node ranges over the exact box test
    const int cx = dir_x(i), cy = dir_y(i), cz = dir_z(i);
    const float dn = nrm.x * cx + nrm.y * cy + nrm.z * cz;
    // nodes u whose segment [u, u + c] (with the offsets) can meet the box
    const int x0 = (int)ceilf(b0.x - DL - BB_EPSX - (float)max(cx, 0)), x1 = (int)floorf(b1.x + DL - BB_EPSX - (float)min(cx, 0));
    const int y0 = (int)ceilf(b0.y - DL - BB_EPSY - (float)max(cy, 0)), y1 = (int)floorf(b1.y + DL - BB_EPSY - (float)min(cy, 0));
    const int z0 = (int)ceilf(b0.z - DL - BB_EPSZ - (float)max(cz, 0)), z1 = (int)floorf(b1.z + DL - BB_EPSZ - (float)min(cz, 0));
    for (int Z = z0; Z <= z1; Z++)
        for (int Y = y0; Y <= y1; Y++) {
            const float syz = nrm.y * (((float)Y + BB_EPSY) - v0.y) + nrm.z * (((float)Z + BB_EPSZ) - v0.z);
            for (int X = x0; X <= x1; X++) {
                const float su = syz + nrm.x * (((float)X + BB_EPSX) - v0.x), sw = su + dn;
                if ((su > tol && sw > tol) || (su < -tol && sw < -tol)) continue;
                // where the link meets the plane must lie in the triangle's box, up to a margin far above the
                // rounding of that point (links almost parallel to the plane go on to the exact test)
                if (fabsf(dn) > tol) {
                    const float s = -su / dn, m = 4.f * tol / fabsf(dn) + 1e-3f;
                    const float px = ((float)X + BB_EPSX) + s * cx, py = ((float)Y + BB_EPSY) + s * cy,
                                pz = ((float)Z + BB_EPSZ) + s * cz;
                    if (px < b0.x - m || px > b1.x + m || py < b0.y - m || py > b1.y + m || pz < b0.z - m ||
                        pz > b1.z + m)
                        continue;
                }
                f(X, Y, Z);
            }
        }
}

template <int G>
__global__ void __launch_bounds__(128) k_link_cand(LbmParams p, DevState d) {
    pdl_wait();
    pdl_trigger();
    const int q = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    const int t = q / G;
    const int grp = q - t * G;
    bool live = t < d.NT;           // every lane stays for the warp's scan below
    float3 v0 = make_float3(0.f, 0.f, 0.f), b0 = v0, b1 = v0, nrm = v0;
    float tol = 0.f;
    if (live) {
        const int k = __float_as_int(d.trec[4 * t + 3].w);
        v0 = f3(d.trec[4 * t]);
        const float3 v1 = f3(d.trec[4 * t + 1]), v2 = f3(d.trec[4 * t + 2]);
        b0 = make_float3(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)));
        b1 = make_float3(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)));
        // the triangles the classification leaves out of its column lists (wider than a column grid, outside
        // their capsule's grid, non-finite) are flagged there and cross nothing here; a triangle as tall as the
        // grid is a broken mesh too.  What is left bounds the loops to CW + 3 nodes per axis.
        const int4 lo = d.cbox[2 * k];
        if (!(b1.x - b0.x < (float)d.CW && b1.y - b0.y < (float)d.CW && b0.x >= (float)(lo.x - 2) &&
              b1.x <= (float)(lo.x + d.CW + 2) && b0.y >= (float)(lo.y - 2) && b1.y <= (float)(lo.y + d.CW + 2))) {
            live = false;
        } else if (!(b1.z - b0.z < (float)d.CW)) {
            atomicOr(d.cnt + 2, 32);
            live = false;
        } else {
            const float3 e1 = sub(v1, v0), e2 = sub(v2, v0);
            // Plane test, conservative: a link whose two ends lie on the same side of the triangle's plane by
            // more than tol (about 1e3 times the rounding of these products) cannot pass seg_tri.
            nrm = cross(e1, e2);
            tol = 1e-3f * (fabsf(e1.x) + fabsf(e1.y) + fabsf(e1.z)) * (fabsf(e2.x) + fabsf(e2.y) + fabsf(e2.z));
        }
    }
    // count, take the warp's places with one atomic, then write (a single counter taking every lane's appends
    // serialises them)
    int n = 0;
    if (live)
        for (int j = 0; j < 9 / G; j++)
            link_candidates(2 * (grp + G * j) + 1, v0, b0, b1, nrm, tol, [&](int, int, int) { n++; });
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int base = 0;
    if (lane == 31 && incl > 0) base = atomicAdd(d.cnt + 7, incl);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - n;
    const int cap = min(d.NT, 1 << 26) * LC_CAP;
    if (live && n > 0)
        for (int j = 0; j < 9 / G; j++) {
            const int i = 2 * (grp + G * j) + 1;
            link_candidates(i, v0, b0, b1, nrm, tol, [&](int X, int Y, int Z) {
                if (base < cap) d.lcand[base] = make_int4(t, X, Y, (Z << 5) | i);
                else atomicOr(d.cnt + 2, 256);
                base++;
            });
        }
}

// One thread per crossing candidate: each end of the link tests the segment as its own search takes it (only in
// its own periodic image; the two segments are the same bits unless rounding at a power of two parts them), and
// the owner field and the list decide which ends record the crossing.
__global__ void __launch_bounds__(128) k_link_test(LbmParams p, DevState d) {
    pdl_wait();
    pdl_trigger();
    const int nc = min(d.cnt[7], min(d.NT, 1 << 26) * LC_CAP);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) {
        const int4 c = d.lcand[q];
        const int t = c.x, X = c.y, Y = c.z, Z = c.w >> 5, i = c.w & 31;
        TriGeom g;
        g.t = t;
        g.k = __float_as_int(d.trec[4 * t + 3].w);
        const float3 v0 = f3(d.trec[4 * t]), v1 = f3(d.trec[4 * t + 1]), v2 = f3(d.trec[4 * t + 2]);
        g.b0 = make_float3(fminf(v0.x, fminf(v1.x, v2.x)), fminf(v0.y, fminf(v1.y, v2.y)), fminf(v0.z, fminf(v1.z, v2.z)));
        g.b1 = make_float3(fmaxf(v0.x, fmaxf(v1.x, v2.x)), fmaxf(v0.y, fmaxf(v1.y, v2.y)), fmaxf(v0.z, fmaxf(v1.z, v2.z)));
        g.v0 = v0;
        g.e1 = sub(v1, v0);
        g.e2 = sub(v2, v0);
        const double* cr = d.cap_red + 4 * g.k;
        g.cr = make_float3((float)cr[1], (float)cr[2], (float)cr[3]);
        const int cx = dir_x(i), cy = dir_y(i), cz = dir_z(i);
        const long long nu = node_of(p, X, Y, Z), nw = node_of(p, X + cx, Y + cy, Z + cz);
        if (nu < 0 || nw < 0) continue;
        float tu = -1.f, tw = -1.f;
        float3 Pu, Du, Pw, Dw;
        const bool iu = own_image(X, g.cr.x, p.nx, true) && own_image(Y, g.cr.y, p.ny, true) &&
                        own_image(Z, g.cr.z, p.nz, !p.walls);
        const bool iw = own_image(X + cx, g.cr.x, p.nx, true) && own_image(Y + cy, g.cr.y, p.ny, true) &&
                        own_image(Z + cz, g.cr.z, p.nz, !p.walls);
        if (iu) {
            end_segment(nu, nw, X, Y, Z, i, Pu, Du);
            tu = seg_cross(g, Pu, Du);
        }
        if (iw) {
            end_segment(nw, nu, X + cx, Y + cy, Z + cz, i + 1, Pw, Dw);
            const bool same = iu && Pw.x == Pu.x && Pw.y == Pu.y && Pw.z == Pu.z && Dw.x == Du.x && Dw.y == Du.y &&
                              Dw.z == Du.z;
            tw = same ? tu : seg_cross(g, Pw, Dw);
        }
        if (tu < 0.f && tw < 0.f) continue;
        // the owners and the list places of both ends, loaded together
        const uint16_t ou = d.owner[nu], ow = d.owner[nw];
        const int bu = d.bidx[nu], bw = d.bidx[nw];
        if (ou == ow || ou == 0xFFFF || ow == 0xFFFF) continue;
        // each end searches the capsule it lies in, else the one across the link
        if (tu >= 0.f && (ou != 0 ? ou : ow) - 1 == g.k) end_record(d, g, bu, i, tu);
        if (tw >= 0.f && (ow != 0 ? ow : ou) - 1 == g.k) end_record(d, g, bw, i + 1, tw);
    }
}

void launch_bb_lists_reset(const DevState& d, cudaStream_t st) {
    if (d.NM == 0) return;
    launch_k(k_lists_reset, dim3(64), dim3(256), 0, st, d);
}

void launch_bb_classify(const LbmParams& p, const DevState& d, int step, bool init, cudaStream_t st) {
    launch_bb_lists_reset(d, st);
    launch_bb_classify_lists(p, d, step, init, st);
}

void launch_bb_classify_lists(const LbmParams& p, const DevState& d, int step, bool init, cudaStream_t st) {
    launch_bb_owner(p, d, step, init, st);
    launch_bb_boundary_list(p, d, st);
}

void launch_bb_owner(const LbmParams& p, const DevState& d, int step, bool init, cudaStream_t st) {
    if (d.NM == 0) return;
    launch_k(k_class_tri, dim3((d.NT + 127) / 128), dim3(128), 0, st, p, d, step);
    launch_k(k_class_col, dim3(box_blocks(d, (size_t)d.CW * d.CW * d.CW), d.NM), dim3(128), 0, st, p, d, init ? 1 : 0);
}

void launch_bb_boundary_list(const LbmParams& p, const DevState& d, cudaStream_t st) {
    if (d.NM == 0) return;
    // boxes are at most CW wide; one node of margin on each side
    const int w = d.CW + 2;
    launch_k(k_boundary_mark, dim3(box_blocks(d, (size_t)w * w * w), d.NM), dim3(128), 0, st, p, d);
    if (d.NT < 65536) launch_k(k_link_cand<9>, dim3(((size_t)d.NT * 9 + 127) / 128), dim3(128), 0, st, p, d);
    else launch_k(k_link_cand<3>, dim3(((size_t)d.NT * 3 + 127) / 128), dim3(128), 0, st, p, d);
    static const int per_t = occupancy((const void*)k_link_test, 128);
    launch_k(k_link_test, dim3(fill_grid(per_t, ((size_t)d.NT * LC_CAP + 127) / 128)), dim3(128), 0, st, p, d);
}

// ------------------------------------------------------------------------------------------------------
// Boundary kernel: collision and streaming of the nodes with cut links
// ------------------------------------------------------------------------------------------------------

// Compile-time loop over the directions: f(std::integral_constant<int, I>) for I = A .. B-1.
template <int A, int B, class F>
__device__ __forceinline__ void for_dirs(F&& f) {
    if constexpr (A < B) {
        f(std::integral_constant<int, A>{});
        for_dirs<A + 1, B>(f);
    }
}

// c_i . v with only the nonzero terms of c_i, in x, y, z order (a product by a zero component is not folded
// away under IEEE rules)
template <int I>
__device__ __forceinline__ float c_dot(float vx, float vy, float vz) {
    float r = 0.f;
    bool first = true;
    auto add = [&](int c, float v) {
        if (c == 0) return;
        const float t = c > 0 ? v : -v;
        r = first ? t : r + t;
        first = false;
    };
    add(dir_x(I), vx);
    add(dir_y(I), vy);
    add(dir_z(I), vz);
    return r;
}

// The lattice neighbourhood of a fluid node: its wrapped coordinates x, y, z and those of x +- 1, y +- 1,
// z +- 1 (z unwrapped between walls, where a fluid node's z +- 1 is in range).
struct Nbhd {
    int x, y, z, xs[3], ys[3], zs[3];   // [1 + c]: coordinate of x + c
    __device__ __forceinline__ Nbhd(const LbmParams& p, int n) {
        z = n / p.nxy;
        const int r = n - z * p.nxy;
        y = r / p.nx;
        x = r - y * p.nx;
        xs[0] = wrapf(x - 1, p.nx); xs[1] = x; xs[2] = wrapf(x + 1, p.nx);
        ys[0] = wrapf(y - 1, p.ny); ys[1] = y; ys[2] = wrapf(y + 1, p.ny);
        zs[0] = p.walls ? z - 1 : wrapf(z - 1, p.nz); zs[1] = z; zs[2] = p.walls ? z + 1 : wrapf(z + 1, p.nz);
    }
    // linear index of x + (cx, cy, cz)
    __device__ __forceinline__ unsigned at(const LbmParams& p, int cx, int cy, int cz) const {
        return (unsigned)xs[1 + cx] + (unsigned)ys[1 + cy] * (unsigned)p.nx + (unsigned)zs[1 + cz] * p.nxy;
    }
};

// The fallback element of a cut link (node x, y, z, direction i) with no crossing: the triangle of capsule cap
// whose centroid is nearest the link's midpoint, lower id on ties; the whole warp searches (warp-convergent
// call), every lane gets the result.
__device__ __forceinline__ int nearest_centroid(const LbmParams& p, const DevState& d, int cap, int x, int y, int z,
                                                int i, int lane) {
    const CapDev cp = d.cap[cap];
    const double* cr = d.cap_red + 4 * cap;
    const float px = near_image(x, (float)cr[1], p.nx, true) + BB_EPSX;
    const float py = near_image(y, (float)cr[2], p.ny, true) + BB_EPSY;
    const float pz = near_image(z, (float)cr[3], p.nz, !p.walls) + BB_EPSZ;
    const float mx = px + 0.5f * dir_x(i), my = py + 0.5f * dir_y(i), mz = pz + 0.5f * dir_z(i);
    float bd = 1e30f;
    int be = -1;
    for (int tl = lane; tl < cp.nt; tl += 32) {
        const int t = cp.t0 + tl;
        const float3 cc = f3(d.trec[4 * t + 3]);
        const float3 dd = make_float3(cc.x - mx, cc.y - my, cc.z - mz);
        const float d2 = dot(dd, dd);
        if (d2 < bd || (d2 == bd && t < be)) { bd = d2; be = t; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float b2 = __shfl_xor_sync(0xffffffffu, bd, o);
        const int e2 = __shfl_xor_sync(0xffffffffu, be, o);
        if (e2 >= 0 && (be < 0 || b2 < bd || (b2 == bd && e2 < be))) { bd = b2; be = e2; }
    }
    return be;
}

// Every boundary node m, one thread each: mean density of its neighbours on the other side of the membrane.
// A node x that sees m across a cut link needs the mean over m's neighbours on x's side (Eq. 14); when m
// borders a single other side that is the same set, so it is computed once per m (otherwise flagged, and
// recomputed per link).
// The same pass settles the element of each of m's cut links for the boundary kernel: the nearest crossing
// the element search recorded, else (no crossing, by round-off) the triangle of the searched capsule whose
// centroid is nearest the link's midpoint, lower id on ties, found by the whole warp.
__global__ void __launch_bounds__(256) k_bb_vrho(LbmParams p, DevState d) {
    pdl_wait();
    pdl_trigger();
    const int nb = min(d.cnt[0], d.maxB);
    const int lane = threadIdx.x & 31;
    // whole warps go round the loop together (the fallback search below takes every lane)
    for (int b0 = blockIdx.x * blockDim.x + threadIdx.x - lane; b0 < nb; b0 += gridDim.x * blockDim.x) {
        const int b = b0 + lane;
        unsigned miss = 0;
        int x = 0, y = 0, z = 0;
        uint16_t me = 0;
        if (b < nb) {
            const int m = d.blist[b];
            const Nbhd nh(p, m);
            x = nh.x; y = nh.y; z = nh.z;
            me = d.owner[m];
            float a = 0.f, c = 0.f, cnt = 0.f;
            int omin = 0x10000, omax = -1;
            for_dirs<1, Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                int e = -1;
                if (!wall_z(p, z + dir_z(i))) {
                    const unsigned q = nh.at(p, dir_x(i), dir_y(i), dir_z(i));
                    const uint16_t oq = d.owner[q];
                    if (oq != 0xFFFF && oq != me) {
                        a += d.rho[q];
                        c += d.rho[p.N + q];
                        cnt += 1.f;
                        omin = min(omin, (int)oq);
                        omax = max(omax, (int)oq);
                        const unsigned long long key = d.bkey[(size_t)b * (Q - 1) + (i - 1)];
                        if (key != ~0ull) e = (int)(unsigned)(key & 0xffffffffull);
                        else miss |= 1u << i;
                    }
                }
                d.belem[(size_t)b * (Q - 1) + (i - 1)] = e;
            });
            d.vrho[m] = make_float4(cnt > 0.f ? a / cnt : 0.f, cnt > 0.f ? c / cnt : 0.f, cnt, omin != omax ? 1.f : 0.f);
        }
        unsigned who = __ballot_sync(0xffffffffu, miss != 0);
        while (who) {
            const int src = __ffs(who) - 1;
            who &= who - 1;
            unsigned mm = __shfl_sync(0xffffffffu, miss, src);
            const int sx = __shfl_sync(0xffffffffu, x, src), sy = __shfl_sync(0xffffffffu, y, src),
                      sz = __shfl_sync(0xffffffffu, z, src), sb = __shfl_sync(0xffffffffu, b, src);
            const int sme = __shfl_sync(0xffffffffu, (int)me, src);
            while (mm) {
                const int i = __ffs(mm) - 1;
                mm &= mm - 1;
                const long long q = node_of(p, sx + dir_x(i), sy + dir_y(i), sz + dir_z(i));
                const int cap = (sme != 0 ? sme : (int)d.owner[q]) - 1;
                const int be = nearest_centroid(p, d, cap, sx, sy, sz, i, lane);
                if (lane == src) {
                    d.belem[(size_t)sb * (Q - 1) + (i - 1)] = be;
                    atomicAdd(d.cnt + 6, 1);
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------------
// Boundary kernel, one thread per boundary node: pull, moments, Shan-Chen force with virtual densities
// across cut links and the wetting offset (Eq. 13-15; reactions to the crossed element), BGK collision,
// streaming with moving half-way bounce-back on walls and cut links (Eq. 11) and the exchanged momentum
// (Eq. 12).
// ------------------------------------------------------------------------------------------------------
// Returns the mass change (A, B) of the node's moving bounce-back links (Eq. 11).
template <typename T>
__device__ __forceinline__ float2 boundary_node(const LbmParams& p, const DevState& d, const T* __restrict__ S,
                                                T* __restrict__ D, const float* __restrict__ ghost, const int step,
                                                int* err, const int b) {
    const int n = d.blist[b];
    const Nbhd nh(p, n);
    const int z = nh.z;
    const uint16_t me = d.owner[n];
    const int pr = step & 1;
    // ---- pull (a deviation storage keeps f - w rref: the reference is added back)
    float fa[Q], fb[Q];
    float ra = 0.f, rb = 0.f;
    for_dirs<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const unsigned src = nh.at(p, -dir_x(i), -dir_y(i), -dir_z(i));
        fa[i] = pld(S + (size_t)i * p.N + src) + dir_w(i) * dev_ref<T>(p, 0);
        fb[i] = pld(S + (size_t)(Q + i) * p.N + src) + dir_w(i) * dev_ref<T>(p, 1);
        ra += fa[i];
        rb += fb[i];
    });
    float jx = 0.f, jy = 0.f, jz = 0.f;
    for_dirs<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float s = fa[i] + fb[i];
        if constexpr (dir_x(i) != 0) jx += dir_x(i) > 0 ? s : -s;
        if constexpr (dir_y(i) != 0) jy += dir_y(i) > 0 ? s : -s;
        if constexpr (dir_z(i) != 0) jz += dir_z(i) > 0 ? s : -s;
    });
    const float pa = psi_fn(ra, p.psi_kind), pb = psi_fn(rb, p.psi_kind);
    // ---- neighbour along c_i: wall (ghost density), same side, or across a cut link (virtual density with the
    // crossed element's colour); the links that bounce back are the cut ones with an element.  In phases, so
    // that each phase's loads are in flight together: the owners; the densities (or, across a cut link, its
    // element and the virtual densities); the elements' colours; then the sums and the reactions.
    uint16_t om[Q];                 // 0xFFFF: a wall plane
    for_dirs<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        om[i] = wall_z(p, z + dir_z(i)) ? (uint16_t)0xFFFF : d.owner[nh.at(p, dir_x(i), dir_y(i), dir_z(i))];
    });
    float va[Q], vb[Q];
    int el[Q];
    unsigned cut = 0, multi = 0;
    for_dirs<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        el[i] = -1;
        if (om[i] == 0xFFFF) {
            const int zn = z + dir_z(i);
            const int w = zn == 0 ? 0 : 1;
            const int rr = nh.xs[1 + dir_x(i)] + nh.ys[1 + dir_y(i)] * p.nx;
            va[i] = ghost[(w * 2 + 0) * p.nxy + rr];
            vb[i] = ghost[(w * 2 + 1) * p.nxy + rr];
        } else {
            const unsigned m = nh.at(p, dir_x(i), dir_y(i), dir_z(i));
            if (om[i] == me) {
                va[i] = d.rho[m];
                vb[i] = d.rho[p.N + m];
            } else {
                el[i] = d.belem[(size_t)b * (Q - 1) + (i - 1)];
                const float4 vr = d.vrho[m];
                va[i] = vr.x;
                vb[i] = vr.y;
                cut |= 1u << i;
                if (vr.w != 0.f) multi |= 1u << i;
            }
        }
    });
    if (multi) {
        // m borders more than one other side: mean over its neighbours on this node's side
        for_dirs<1, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            if (!((multi >> i) & 1u)) return;
            const Nbhd mh(p, (int)nh.at(p, dir_x(i), dir_y(i), dir_z(i)));
            float sA = 0.f, sB = 0.f;
            int cnt = 0;
            for (int q = 1; q < Q; q++) {
                if (wall_z(p, mh.z + dir_z(q))) continue;
                const unsigned qq = mh.at(p, dir_x(q), dir_y(q), dir_z(q));
                if (d.owner[qq] != me) continue;
                sA += d.rho[qq];
                sB += d.rho[p.N + qq];
                cnt++;
            }
            va[i] = cnt ? sA / cnt : ra;
            vb[i] = cnt ? sB / cnt : rb;
        });
    }
    // the crossed element's colour (per capsule or per element) on the virtual density: an offset of
    // |colour| (rho_maj - rho_min) / 2 (Eq. 15 with its normalisation read so that Sec. III.D's contact angles
    // hold, cos theta = colour)
    const float drho = (float)(d.rho_maj - d.rho_min);
    for_dirs<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        if (!((cut >> i) & 1u) || el[i] < 0) return;
        const float col = d.tcol[el[i]];
        const float rv = 0.5f * fabsf(col) * drho;
        if (col > 0.f) va[i] += rv;
        else if (col < 0.f) vb[i] += rv;
    });
    float sa0 = 0.f, sa1 = 0.f, sa2 = 0.f, sb0 = 0.f, sb1 = 0.f, sb2 = 0.f;
    unsigned bounce = 0;
    for_dirs<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr float wi = dir_w(i);
        float psA = 0.f, psB = 0.f;
        if (!((cut >> i) & 1u)) {
            psA = psi_fn(va[i], p.psi_kind);
            psB = psi_fn(vb[i], p.psi_kind);
        } else if (el[i] >= 0) {
            psA = psi_fn(va[i], p.psi_kind);
            psB = psi_fn(vb[i], p.psi_kind);
            // reaction of both components on the element: + psi^c(x) G w_i psi^{c'}(virtual) c_i
            const float a = p.G * wi * (pa * psB + pb * psA);
            atomicAdd(&d.epend[pr * d.NT + el[i]], make_float4(a * dir_x(i), a * dir_y(i), a * dir_z(i), 0.f));
            bounce |= 1u << i;
        } else {
            atomicOr(err, 2);      // list out of step with the owner field: never expected
        }
        const float qa = wi * psA, qb = wi * psB;
        if constexpr (dir_x(i) != 0) { sa0 += dir_x(i) > 0 ? qa : -qa; sb0 += dir_x(i) > 0 ? qb : -qb; }
        if constexpr (dir_y(i) != 0) { sa1 += dir_y(i) > 0 ? qa : -qa; sb1 += dir_y(i) > 0 ? qb : -qb; }
        if constexpr (dir_z(i) != 0) { sa2 += dir_z(i) > 0 ? qa : -qa; sb2 += dir_z(i) > 0 ? qb : -qb; }
    });
    const float FA[3] = {-pa * p.G * sb0 + ra * p.g[0], -pa * p.G * sb1 + ra * p.g[1], -pa * p.G * sb2 + ra * p.g[2]};
    const float FB[3] = {-pb * p.G * sa0 + rb * p.g[0], -pb * p.G * sa1 + rb * p.g[1], -pb * p.G * sa2 + rb * p.g[2]};
    const float rt = ra + rb, irt = 1.f / rt;
    const float ux = jx * irt, uy = jy * irt, uz = jz * irt;
    if (!(rt > 0.f) || !(ux * ux + uy * uy + uz * uz <= 0.09f)) atomicOr(err, 1);
    const float ta = ra > 0.f ? p.tau / ra : 0.f, tb = rb > 0.f ? p.tau / rb : 0.f;
    const float uA[3] = {ux + ta * FA[0], uy + ta * FA[1], uz + ta * FA[2]};
    const float uB[3] = {ux + tb * FB[0], uy + tb * FB[1], uz + tb * FB[2]};
    const float uuA = uA[0] * uA[0] + uA[1] * uA[1] + uA[2] * uA[2];
    const float uuB = uB[0] * uB[0] + uB[1] * uB[1] + uB[2] * uB[2];
    // ---- equilibrium (Eq. 2) and collision; the rest population closes the mass
    float sA = 0.f, sB = 0.f;
    for_dirs<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr float wi = dir_w(i);
        const float cuA = c_dot<i>(uA[0], uA[1], uA[2]), cuB = c_dot<i>(uB[0], uB[1], uB[2]);
        const float eA = wi * ra * (1.f + 3.f * cuA + 4.5f * cuA * cuA - 1.5f * uuA);
        const float eB = wi * rb * (1.f + 3.f * cuB + 4.5f * cuB * cuB - 1.5f * uuB);
        sA += eA;
        sB += eB;
        fa[i] = fa[i] + p.omega * (eA - fa[i]);
        fb[i] = fb[i] + p.omega * (eB - fb[i]);
    });
    fa[0] = fa[0] + p.omega * ((ra - sA) - fa[0]);
    fb[0] = fb[0] + p.omega * ((rb - sB) - fb[0]);
    // ---- streaming (a deviation storage keeps f - w rref; opposite directions share their weight)
    float dmA = 0.f, dmB = 0.f;
    pst(D + n, fa[0] - dir_w(0) * dev_ref<T>(p, 0));
    pst(D + (size_t)Q * p.N + n, fb[0] - dir_w(0) * dev_ref<T>(p, 1));
    for_dirs<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int io = dir_opp(i);
        const float gA = dir_w(i) * dev_ref<T>(p, 0), gB = dir_w(i) * dev_ref<T>(p, 1);
        const float oA = fa[i], oB = fb[i];
        const int zn = z + dir_z(i);
        if (wall_z(p, zn)) {
            const float* U = zn == 0 ? p.ulo : p.uhi;
            const float cU = 6.f * dir_w(i) * (dir_x(i) * U[0] + dir_y(i) * U[1] + dir_z(i) * U[2]);
            const unsigned tgt = (unsigned)(nh.xs[1 + dir_x(i)] + nh.ys[1 + dir_y(i)] * p.nx) + (unsigned)zn * p.nxy;
            pst(D + (size_t)io * p.N + tgt, oA - cU * ra - gA);
            pst(D + (size_t)(Q + io) * p.N + tgt, oB - cU * rb - gB);
        } else if (!((bounce >> i) & 1u)) {
            pst(D + (size_t)i * p.N + n, oA - gA);
            pst(D + (size_t)(Q + i) * p.N + n, oB - gB);
        } else {
            // moving half-way bounce-back (Eq. 11) with the element velocity; exchanged momentum (Eq. 12)
            const unsigned m = nh.at(p, dir_x(i), dir_y(i), dir_z(i));
            const int e = el[i];
            const int4 Te = d.tri[e];
            const float4 V0 = d.V[Te.x], V1 = d.V[Te.y], V2 = d.V[Te.z];
            const float vx = (V0.x + V1.x + V2.x) * (1.f / 3.f), vy = (V0.y + V1.y + V2.y) * (1.f / 3.f),
                        vz = (V0.z + V1.z + V2.z) * (1.f / 3.f);
            const float cv = 6.f * dir_w(i) * (dir_x(i) * vx + dir_y(i) * vy + dir_z(i) * vz);
            const float bA = oA - cv * ra, bB = oB - cv * rb;
            pst(D + (size_t)io * p.N + m, bA - gA);
            pst(D + (size_t)(Q + io) * p.N + m, bB - gB);
            const float dp = oA + bA + oB + bB;
            atomicAdd(&d.emom[pr * d.NT + e], make_float4(dp * dir_x(i), dp * dir_y(i), dp * dir_z(i), 0.f));
            dmA += bA - oA;
            dmB += bB - oB;
        }
    });
    return make_float2(dmA, dmB);
}

// Grid-stride over the boundary list, a thread per node; each block writes the sum of its nodes' mass changes,
// in a fixed order, to bdm[blockIdx.x] and block 0 records the number of partials.
constexpr int BT_THREADS = 128;

template <typename T>
__global__ void __launch_bounds__(BT_THREADS) k_boundary(LbmParams p, DevState d, const T* __restrict__ S,
                                                         T* __restrict__ D, const float* __restrict__ ghost,
                                                         int step, int* err) {
    pdl_wait();
    pdl_trigger();
    __shared__ float2 part[BT_THREADS / 32];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = min(d.cnt[0], d.maxB);
    float2 acc = make_float2(0.f, 0.f);
    for (int b = blockIdx.x * BT_THREADS + threadIdx.x; b < nb; b += gridDim.x * BT_THREADS) {
        const float2 v = boundary_node<T>(p, d, S, D, ghost, step, err, b);
        acc.x += v.x;
        acc.y += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) part[wl] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = part[0];
        for (int w = 1; w < BT_THREADS / 32; w++) { t.x += part[w].x; t.y += part[w].y; }
        d.bdm[blockIdx.x] = t;
        if (blockIdx.x == 0) d.cnt[5] = (int)gridDim.x;
    }
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// k_bb_vrho with one warp per node, lane i-1 looking at direction i (the short-list form, beside
// k_boundary_warp).
__global__ void __launch_bounds__(256) k_bb_vrho_warp(LbmParams p, DevState d) {
    pdl_wait();
    pdl_trigger();
    const int nb = min(d.cnt[0], d.maxB);
    const int lane = threadIdx.x & 31;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += (gridDim.x * blockDim.x) >> 5) {
        const int m = d.blist[b];
        const int z = m / p.nxy, r = m - z * p.nxy, y = r / p.nx, x = r - y * p.nx;
        const uint16_t me = d.owner[m];
        float a = 0.f, c = 0.f, cnt = 0.f;
        int omin = 0x10000, omax = -1;
        int e = -1, my_cap = -1;
        if (lane < Q - 1) {
            const int i = lane + 1;
            const long long q = node_of(p, x + dir_x(i), y + dir_y(i), z + dir_z(i));
            if (q >= 0) {
                const uint16_t oq = d.owner[q];
                if (oq != 0xFFFF && oq != me) {
                    a = d.rho[q];
                    c = d.rho[p.N + q];
                    cnt = 1.f;
                    omin = omax = oq;
                    my_cap = (me != 0 ? me : oq) - 1;
                    const unsigned long long key = d.bkey[(size_t)b * (Q - 1) + lane];
                    if (key != ~0ull) e = (int)(unsigned)(key & 0xffffffffull);
                }
            }
        }
        a = wsum(a);
        c = wsum(c);
        cnt = wsum(cnt);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            omin = min(omin, __shfl_xor_sync(0xffffffffu, omin, o));
            omax = max(omax, __shfl_xor_sync(0xffffffffu, omax, o));
        }
        if (lane == 0)
            d.vrho[m] = make_float4(cnt > 0.f ? a / cnt : 0.f, cnt > 0.f ? c / cnt : 0.f, cnt, omin != omax ? 1.f : 0.f);
        unsigned mm = __ballot_sync(0xffffffffu, my_cap >= 0 && e < 0);
        while (mm) {
            const int li = __ffs(mm) - 1;
            mm &= mm - 1;
            const int i = li + 1;
            const int cap = __shfl_sync(0xffffffffu, my_cap, li);
            const int be = nearest_centroid(p, d, cap, x, y, z, i, lane);
            if (lane == li) {
                e = be;
                atomicAdd(d.cnt + 6, 1);
            }
        }
        if (lane < Q - 1) d.belem[(size_t)b * (Q - 1) + lane] = e;
    }
}

// The same boundary update with one warp per node, lane i owning direction i (i = 0..18), moments and force sums
// by warp reductions: each node's links run side by side, which suits short lists (a few capsules), where the
// thread-per-node form leaves most SMs idle and each thread waits through its links one after another.
// Returns the mass change (A, B) of the node's moving bounce-back links (Eq. 11), in every lane.
template <typename T>
__device__ __forceinline__ float2 boundary_node_warp(const LbmParams& p, const DevState& d, const T* __restrict__ S,
                                                T* __restrict__ D, const float* __restrict__ ghost, const int step,
                                                int* err, const int b, const int lane) {
    const int n = d.blist[b];
    const int z = n / p.nxy, r = n - z * p.nxy, y = r / p.nx, x = r - y * p.nx;
    const uint16_t me = d.owner[n];
    const int i = lane < Q ? lane : 0;
    const bool dl = lane < Q;                         // lanes carrying a direction
    const int cx = dir_x(i), cy = dir_y(i), cz = dir_z(i);
    const float wi = dir_w(i);
    const int pr = step & 1;
    // ---- pull
    float fa = 0.f, fb = 0.f;
    if (dl) {
        int zs = z - cz;
        if (!p.walls) zs = wrapf(zs, p.nz);
        const unsigned int src = (unsigned)wrapf(x - cx, p.nx) + (unsigned)wrapf(y - cy, p.ny) * p.nx + (unsigned)zs * p.nxy;
        fa = pld(S + (size_t)i * p.N + src) + wi * dev_ref<T>(p, 0);      // + the reference of a deviation storage
        fb = pld(S + (size_t)(Q + i) * p.N + src) + wi * dev_ref<T>(p, 1);
    }
    const float ra = wsum(fa), rb = wsum(fb);
    const float jx = wsum(cx * (fa + fb)), jy = wsum(cy * (fa + fb)), jz = wsum(cz * (fa + fb));
    const float pa = psi_fn(ra, p.psi_kind), pb = psi_fn(rb, p.psi_kind);
    // ---- neighbour along c_i: wall, same side, or across a cut link
    const int zn = z + cz;
    const bool wall = dl && lane > 0 && wall_z(p, zn);
    long long m = -1;
    uint16_t om = me;
    int e = -1;
    float psA = 0.f, psB = 0.f;
    if (dl && lane > 0) {
        if (wall) {
            const int w = zn == 0 ? 0 : 1;
            const int rr = wrapf(x + cx, p.nx) + wrapf(y + cy, p.ny) * p.nx;
            psA = psi_fn(ghost[(w * 2 + 0) * p.nxy + rr], p.psi_kind);
            psB = psi_fn(ghost[(w * 2 + 1) * p.nxy + rr], p.psi_kind);
        } else {
            m = node_of(p, x + cx, y + cy, zn);
            om = d.owner[m];
            if (om == me) {
                psA = psi_fn(d.rho[m], p.psi_kind);
                psB = psi_fn(d.rho[p.N + m], p.psi_kind);
            } else {
                e = d.belem[(size_t)b * (Q - 1) + lane - 1];
                float vA, vB;
                const float4 vr = d.vrho[m];
                if (vr.w == 0.f) {
                    vA = vr.x;
                    vB = vr.y;
                } else {
                    // m borders more than one other side: mean over its neighbours on this node's side
                    const int mz = (int)(m / p.nxy), mr = (int)(m - (long long)mz * p.nxy), my = mr / p.nx,
                              mx = mr - my * p.nx;
                    float sA = 0.f, sB = 0.f;
                    int cnt = 0;
                    for (int q = 1; q < Q; q++) {
                        const long long qq = node_of(p, mx + dir_x(q), my + dir_y(q), mz + dir_z(q));
                        if (qq < 0) continue;
                        const uint16_t oq = d.owner[qq];
                        if (oq == 0xFFFF || oq != me) continue;
                        sA += d.rho[qq];
                        sB += d.rho[p.N + qq];
                        cnt++;
                    }
                    vA = cnt ? sA / cnt : ra;
                    vB = cnt ? sB / cnt : rb;
                }
                if (e >= 0) {
                    const float col = d.tcol[e];     // the crossed element's colour (per capsule or per element)
                    const float rv = 0.5f * fabsf(col) * (float)(d.rho_maj - d.rho_min);
                    if (col > 0.f) vA += rv;
                    else if (col < 0.f) vB += rv;
                    psA = psi_fn(vA, p.psi_kind);
                    psB = psi_fn(vB, p.psi_kind);
                    // reaction of both components on the element: + psi^c(x) G w_i psi^{c'}(virtual) c_i
                    const float a = p.G * wi * (pa * psB + pb * psA);
                    atomicAdd(&d.epend[pr * d.NT + e], make_float4(a * cx, a * cy, a * cz, 0.f));
                } else {
                    atomicOr(err, 2);      // list out of step with the owner field: never expected
                }
            }
        }
    }
    const float qa = wi * psA, qb = wi * psB;
    const float sa0 = wsum(qa * cx), sa1 = wsum(qa * cy), sa2 = wsum(qa * cz);
    const float sb0 = wsum(qb * cx), sb1 = wsum(qb * cy), sb2 = wsum(qb * cz);
    const float FA[3] = {-pa * p.G * sb0 + ra * p.g[0], -pa * p.G * sb1 + ra * p.g[1], -pa * p.G * sb2 + ra * p.g[2]};
    const float FB[3] = {-pb * p.G * sa0 + rb * p.g[0], -pb * p.G * sa1 + rb * p.g[1], -pb * p.G * sa2 + rb * p.g[2]};
    const float rt = ra + rb, irt = 1.f / rt;
    const float ux = jx * irt, uy = jy * irt, uz = jz * irt;
    if (lane == 0 && (!(rt > 0.f) || !(ux * ux + uy * uy + uz * uz <= 0.09f))) atomicOr(err, 1);
    const float ta = ra > 0.f ? p.tau / ra : 0.f, tb = rb > 0.f ? p.tau / rb : 0.f;
    const float uA[3] = {ux + ta * FA[0], uy + ta * FA[1], uz + ta * FA[2]};
    const float uB[3] = {ux + tb * FB[0], uy + tb * FB[1], uz + tb * FB[2]};
    // ---- equilibrium (Eq. 2) of this lane's direction; the rest population closes the mass
    float eA = 0.f, eB = 0.f;
    if (dl && lane > 0) {
        const float cuA = cx * uA[0] + cy * uA[1] + cz * uA[2];
        const float cuB = cx * uB[0] + cy * uB[1] + cz * uB[2];
        const float uuA = uA[0] * uA[0] + uA[1] * uA[1] + uA[2] * uA[2];
        const float uuB = uB[0] * uB[0] + uB[1] * uB[1] + uB[2] * uB[2];
        eA = wi * ra * (1.f + 3.f * cuA + 4.5f * cuA * cuA - 1.5f * uuA);
        eB = wi * rb * (1.f + 3.f * cuB + 4.5f * cuB * cuB - 1.5f * uuB);
    }
    const float sA = wsum(eA), sB = wsum(eB);
    if (lane == 0) { eA = ra - sA; eB = rb - sB; }
    const float oA = fa + p.omega * (eA - fa), oB = fb + p.omega * (eB - fb);
    // ---- streaming (a deviation storage keeps f - w rref; opposite directions share their weight)
    float dm[2] = {0.f, 0.f};
    const float gA = wi * dev_ref<T>(p, 0), gB = wi * dev_ref<T>(p, 1);
    if (dl) {
        if (lane == 0) {
            pst(D + n, oA - gA);
            pst(D + (size_t)Q * p.N + n, oB - gB);
        } else if (wall) {
            const float* U = zn == 0 ? p.ulo : p.uhi;
            const float cU = 6.f * wi * (cx * U[0] + cy * U[1] + cz * U[2]);
            const unsigned int tgt = (unsigned)(wrapf(x + cx, p.nx) + wrapf(y + cy, p.ny) * p.nx) + (unsigned)zn * p.nxy;
            pst(D + (size_t)dir_opp(i) * p.N + tgt, oA - cU * ra - gA);
            pst(D + (size_t)(Q + dir_opp(i)) * p.N + tgt, oB - cU * rb - gB);
        } else if (om == me || e < 0) {
            pst(D + (size_t)i * p.N + n, oA - gA);
            pst(D + (size_t)(Q + i) * p.N + n, oB - gB);
        } else {
            // moving half-way bounce-back (Eq. 11) with the element velocity; exchanged momentum (Eq. 12)
            const int4 tv = d.tri[e];
            const float4 V0 = d.V[tv.x], V1 = d.V[tv.y], V2 = d.V[tv.z];
            const float vx = (V0.x + V1.x + V2.x) * (1.f / 3.f), vy = (V0.y + V1.y + V2.y) * (1.f / 3.f),
                        vz = (V0.z + V1.z + V2.z) * (1.f / 3.f);
            const float cv = 6.f * wi * (cx * vx + cy * vy + cz * vz);
            const float bA = oA - cv * ra, bB = oB - cv * rb;
            pst(D + (size_t)dir_opp(i) * p.N + m, bA - gA);
            pst(D + (size_t)(Q + dir_opp(i)) * p.N + m, bB - gB);
            const float dp = oA + bA + oB + bB;
            atomicAdd(&d.emom[pr * d.NT + e], make_float4(dp * cx, dp * cy, dp * cz, 0.f));
            dm[0] = bA - oA;
            dm[1] = bB - oB;
        }
    }
    return make_float2(wsum(dm[0]), wsum(dm[1]));
}

// Grid-stride over the boundary list, 8 warps per block; each block writes the sum of its nodes' mass
// changes, in a fixed order, to bdm[blockIdx.x] and block 0 records the number of partials.
template <typename T>
__global__ void __launch_bounds__(256) k_boundary_warp(LbmParams p, DevState d, const T* __restrict__ S,
                                                  T* __restrict__ D, const float* __restrict__ ghost,
                                                  int step, int* err) {
    pdl_wait();
    pdl_trigger();
    __shared__ float2 part[8];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = min(d.cnt[0], d.maxB);
    float2 acc = make_float2(0.f, 0.f);
    for (int b = blockIdx.x * 8 + wl; b < nb; b += gridDim.x * 8) {
        const float2 v = boundary_node_warp<T>(p, d, S, D, ghost, step, err, b, lane);
        acc.x += v.x;
        acc.y += v.y;
    }
    if (lane == 0) part[wl] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = part[0];
        for (int w = 1; w < 8; w++) { t.x += part[w].x; t.y += part[w].y; }
        d.bdm[blockIdx.x] = t;
        if (blockIdx.x == 0) d.cnt[5] = (int)gridDim.x;
    }
}

// A list of this capacity or more takes the thread-per-node forms, a shorter one the warp-per-node forms
// (SCBB_BOUNDARY_FORM=warp or thread forces one).
constexpr int THREAD_FORM_NODES = 65536;
static bool thread_form(const DevState& d) {
    static const int force = [] {
        const char* e = getenv("SCBB_BOUNDARY_FORM");
        if (e && !strcmp(e, "warp")) return 0;
        if (e && !strcmp(e, "thread")) return 1;
        return -1;
    }();
    return force >= 0 ? force == 1 : d.maxB >= THREAD_FORM_NODES;
}

void launch_bb_vrho(const LbmParams& p, const DevState& d, cudaStream_t st) {
    if (d.NM == 0) return;
    if (thread_form(d)) {
        const size_t need = ((size_t)d.maxB + 255) / 256;
        static const int per_v = occupancy((const void*)k_bb_vrho, 256);
        launch_k(k_bb_vrho, dim3(fill_grid(per_v, need)), dim3(256), 0, st, p, d);
    } else {
        const size_t need = ((size_t)d.maxB + 7) / 8;
        static const int per_v = occupancy((const void*)k_bb_vrho_warp, 256);
        launch_k(k_bb_vrho_warp, dim3(fill_grid(per_v, need)), dim3(256), 0, st, p, d);
    }
}

void launch_bb_boundary(const LbmParams& p, const DevState& d, const float* S, float* D, const float* ghost,
                        int step, int* err, cudaStream_t st) {
    if (d.NM == 0) return;
    launch_bb_vrho(p, d, st);
    with_storage(p.store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        if (thread_form(d)) {
            const size_t need = ((size_t)d.maxB + BT_THREADS - 1) / BT_THREADS;   // the partials fit in bdm[maxB]
            static const int per_b = occupancy((const void*)k_boundary<T>, BT_THREADS);
            launch_k(k_boundary<T>, dim3(fill_grid(per_b, need)), dim3(BT_THREADS), 0, st, p, d,
                     reinterpret_cast<const T*>(S), reinterpret_cast<T*>(D), ghost, step, err);
        } else {
            const size_t need = ((size_t)d.maxB + 7) / 8;   // 8 warps per block; the partials fit in bdm[maxB]
            static const int per_b = occupancy((const void*)k_boundary_warp<T>, 256);
            launch_k(k_boundary_warp<T>, dim3(fill_grid(per_b, need)), dim3(256), 0, st, p, d,
                     reinterpret_cast<const T*>(S), reinterpret_cast<T*>(D), ghost, step, err);
        }
    });
}

// ------------------------------------------------------------------------------------------------------
// Fresh nodes
// ------------------------------------------------------------------------------------------------------

// Mass of the state before the fresh update and the correction factors of Eq. 18.  Collision and streaming
// conserve each component's mass exactly, so M(t) - M(0) is the running FP64 sum of the changes the method
// makes on purpose: the moving bounce-back of every boundary node of this step (Eq. 11) and the fresh-node
// replacements of the previous step (Eq. 16).  Summing M(t) over the FP32 lattice instead would carry its
// rounding (systematic over uniform regions), which Eq. 18 multiplies by C0 sum(rho_init)/rho_init^c.
__global__ void __launch_bounds__(1024) k_mass_finalize(DevState d, double vsys) {
    pdl_wait();
    pdl_trigger();
    // the changes are small: FP32 partials per thread and per warp, FP64 only in warp 0
    __shared__ float shf[2][32];
    float fa = 0.f, fb = 0.f;
    const int nb = min(d.cnt[5], d.maxB);            // block partials of this step's boundary kernel
    const int nf = min(d.cnt[4], d.maxF);
#pragma unroll 4
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        const float2 v = d.bdm[q];
        fa += v.x;
        fb += v.y;
    }
    for (int q = threadIdx.x; q < nf; q += blockDim.x) {
        const float2 v = d.fdm[q];
        fa += v.x;
        fb += v.y;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fa += __shfl_xor_sync(0xffffffffu, fa, o);
        fb += __shfl_xor_sync(0xffffffffu, fb, o);
    }
    if (lane == 0) { shf[0][w] = fa; shf[1][w] = fb; }
    __syncthreads();
    if (w == 0) {
        double a = lane < (int)(blockDim.x >> 5) ? (double)shf[0][lane] : 0.0;
        double b = lane < (int)(blockDim.x >> 5) ? (double)shf[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            const double dM[2] = {d.mass[2] + a, d.mass[3] + b};
            const double ri[2] = {d.mass[0] / vsys, d.mass[1] / vsys};
            for (int c = 0; c < 2; c++) {
                d.mass[2 + c] = dM[c];
                d.mass[4 + c] = d.mass_correction ? 1.0 - d.C0 * (ri[0] + ri[1]) / ri[c] * dM[c] / vsys : 1.0;
            }
        }
    }
}

// density of node m of the new state (pull from S)
template <typename T>
__device__ __forceinline__ void pulled_rho(const LbmParams& p, const T* __restrict__ S, int m, float& ra, float& rb) {
    const int z = m / p.nxy, r = m - z * p.nxy, y = r / p.nx, x = r - y * p.nx;
    Cols k;
    k.cx[0] = wrapf(x - 1, p.nx); k.cx[1] = x; k.cx[2] = wrapf(x + 1, p.nx);
    k.ry[0] = wrapf(y - 1, p.ny) * p.nx; k.ry[1] = y * p.nx; k.ry[2] = wrapf(y + 1, p.ny) * p.nx;
    float f[2 * Q];
    pull(p, S, k, z, f);
    ra = rb = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) { ra += f[i]; rb += f[Q + i]; }
}

// One warp per fresh node: lanes 0-17 pull the densities of the 18 neighbours, then the warp scans the
// capsule's triangle centroids for the nearest element.
template <typename T>
__device__ __forceinline__ void fresh_node(const LbmParams& p, const DevState& d, const T* __restrict__ S, const int q,
                                           const int lane, int* queue) {
    const int n = d.flist[q];
    const int z = n / p.nxy, r = n - z * p.nxy, y = r / p.nx, x = r - y * p.nx;
    const uint16_t side = d.owner[n];
    // this lane's neighbour (direction lane + 1): same side? fresh? its density
    bool same = false, fr = false;
    float a = 0.f, b = 0.f;
    if (lane < Q - 1) {
        const int i = lane + 1;
        const long long m = node_of(p, x + dir_x(i), y + dir_y(i), z + dir_z(i));
        if (m >= 0 && d.owner[m] == side) {
            same = true;
            fr = (d.fmask[m >> 5] >> (m & 31)) & 1u;
            pulled_rho(p, S, (int)m, a, b);
        }
    }
    float rf[2] = {0.f, 0.f};
    bool ok = false;
    for (int pass = 0; pass < 2 && !ok; pass++) {
        const bool use = same && (pass == 1 || !fr);
        float sum0 = use ? a : 0.f, sum1 = use ? b : 0.f;
        float mn0 = use ? a : 1e30f, mn1 = use ? b : 1e30f, mx0 = use ? a : -1e30f, mx1 = use ? b : -1e30f;
        int cnt = use ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum0 += __shfl_xor_sync(0xffffffffu, sum0, o);
            sum1 += __shfl_xor_sync(0xffffffffu, sum1, o);
            mn0 = fminf(mn0, __shfl_xor_sync(0xffffffffu, mn0, o));
            mn1 = fminf(mn1, __shfl_xor_sync(0xffffffffu, mn1, o));
            mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
            mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        }
        if (cnt) {
            rf[0] = fminf(fmaxf(sum0 / cnt * (float)d.mass[4], mn0), mx0);
            rf[1] = fminf(fmaxf(sum1 / cnt * (float)d.mass[5], mn1), mx1);
            ok = true;
        }
    }
    if (!ok) {
        if (lane == 0) d.fnew[2 * q] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    // nearest element (centroid) of the capsule that moved over the node
    const int cap = (side != 0 ? side : d.fold[q]) - 1;
    const CapDev cp = d.cap[cap];
    const double* cr = d.cap_red + 4 * cap;
    const float px = near_image(x, (float)cr[1], p.nx, true), py = near_image(y, (float)cr[2], p.ny, true);
    const float pz = near_image(z, (float)cr[3], p.nz, !p.walls);
    float bd = 1e30f;
    int be = -1;
    // Candidates within distance r of the node, r = 1 then 2: a triangle's centroid lies inside its own
    // bounding box, so every centroid within r is listed in the (2r+1) x (2r+1) column cells around the
    // node and its box meets the cube of half-width r around the node.  A nearest centroid found within r
    // is therefore the nearest of the whole capsule (ties included); a node the membrane has just swept
    // over almost always has one within 1.  Otherwise scan the whole capsule.
    const int4 lo = d.cbox[2 * cap];
    const int ccx = (int)floorf(px) - lo.x, ccy = (int)floorf(py) - lo.y;
    for (int r = 1; r <= 2; r++) {
        const float fr = (float)r;
        const CellScan cs = cell_scan(d, cap, ccx - r, ccy - r, 2 * r + 1, lane);
        for_candidates(d, cs, make_float3(px - fr, py - fr, pz - fr), make_float3(px + fr, py + fr, pz + fr),
                       queue, lane, [&](int t) {
                           if (t < 0) return;
                           const float3 c = f3(d.trec[4 * t + 3]);
                           const float dx = c.x - px, dy = c.y - py, dz = c.z - pz;
                           const float d2 = dx * dx + dy * dy + dz * dz;
                           if (d2 < bd || (d2 == bd && t < be)) { bd = d2; be = t; }
                       });
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float b2 = __shfl_xor_sync(0xffffffffu, bd, o);
            const int e2 = __shfl_xor_sync(0xffffffffu, be, o);
            if (e2 >= 0 && (be < 0 || b2 < bd || (b2 == bd && e2 < be))) { bd = b2; be = e2; }
        }
        if (bd <= fr * fr) break;
    }
    if (!(bd <= 4.f)) {
        bd = 1e30f;
        be = -1;
        for (int tl = lane; tl < cp.nt; tl += 32) {
            const int t = cp.t0 + tl;
            const float3 c = f3(d.trec[4 * t + 3]);
            const float dx = c.x - px, dy = c.y - py, dz = c.z - pz;
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < bd) { bd = d2; be = t; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float b2 = __shfl_xor_sync(0xffffffffu, bd, o);
            const int e2 = __shfl_xor_sync(0xffffffffu, be, o);
            if (e2 >= 0 && (be < 0 || b2 < bd || (b2 == bd && e2 < be))) { bd = b2; be = e2; }
        }
    }
    if (be < 0) {                                  // no finite distance (non-finite geometry): keep the node
        if (lane == 0) {
            d.fnew[2 * q] = make_float4(0.f, 0.f, 0.f, 0.f);
            atomicOr(d.cnt + 2, 128);
        }
        return;
    }
    if (lane == 0) {
        const int4 tv = d.tri[be];
        const float3 v = make_float3((d.V[tv.x].x + d.V[tv.y].x + d.V[tv.z].x) * (1.f / 3.f),
                                     (d.V[tv.x].y + d.V[tv.y].y + d.V[tv.z].y) * (1.f / 3.f),
                                     (d.V[tv.x].z + d.V[tv.y].z + d.V[tv.z].z) * (1.f / 3.f));
        d.fnew[2 * q] = make_float4(rf[0], rf[1], 1.f, 0.f);
        d.fnew[2 * q + 1] = make_float4(v.x, v.y, v.z, __int_as_float(be));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fresh_compute(LbmParams p, DevState d, const T* __restrict__ S) {
    pdl_wait();
    pdl_trigger();
    __shared__ int queue[8][CAND_Q];
    const int nf = min(d.cnt[1], d.maxF);
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nf; q += (gridDim.x * blockDim.x) >> 5) {
        fresh_node<T>(p, d, S, q, threadIdx.x & 31, queue[threadIdx.x >> 5]);
        __syncwarp();
    }
}

// Writes f_eq(rho_fresh, v) into the slots the fresh node pulls from (Eq. 2, 16-18) and hands the element
// the removed minus the created momentum.
template <typename T>
__device__ __forceinline__ void fresh_apply_node(const LbmParams& p, const DevState& d, T* __restrict__ S,
                                                 const int step, const int q) {
    const float4 a = d.fnew[2 * q];
    if (a.z == 0.f) {
        d.fdm[q] = make_float2(0.f, 0.f);          // populations kept
        return;
    }
    const float4 vv = d.fnew[2 * q + 1];
    const int e = __float_as_int(vv.w);
    const int n = d.flist[q];
    const int z = n / p.nxy, r = n - z * p.nxy, y = r / p.nx, x = r - y * p.nx;
    Cols k;
    k.cx[0] = wrapf(x - 1, p.nx); k.cx[1] = x; k.cx[2] = wrapf(x + 1, p.nx);
    k.ry[0] = wrapf(y - 1, p.ny) * p.nx; k.ry[1] = y * p.nx; k.ry[2] = wrapf(y + 1, p.ny) * p.nx;
    int zm = z - 1, zp = z + 1;
    if (!p.walls) { zm = wrapf(zm, p.nz); zp = wrapf(zp, p.nz); }
    const int pz[3] = {zm * p.nxy, z * p.nxy, zp * p.nxy};
    const float uu = vv.x * vv.x + vv.y * vv.y + vv.z * vv.z;
    float rem[3] = {0.f, 0.f, 0.f};
    float dA = 0.f, dB = 0.f;                      // mass change of the replacement, per component
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const unsigned int m = k.cx[1 - dir_x(i)] + k.ry[1 - dir_y(i)] + pz[1 - dir_z(i)];
        const float cu = dir_x(i) * vv.x + dir_y(i) * vv.y + dir_z(i) * vv.z;
        const float e0 = dir_w(i) * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * uu);
        T* sa = S + (size_t)i * p.N + m;
        T* sb = S + (size_t)(Q + i) * p.N + m;
        // a deviation storage keeps f - w_i rref^c: the reference is added on the load and taken off the store
        const float ga = dir_w(i) * dev_ref<T>(p, 0), gb = dir_w(i) * dev_ref<T>(p, 1);
        const float oa = pldc(sa) + ga, ob = pldc(sb) + gb;
        const float old = oa + ob;
        rem[0] += dir_x(i) * old; rem[1] += dir_y(i) * old; rem[2] += dir_z(i) * old;
        const float sna = pround(e0 * a.x - ga, S), snb = pround(e0 * a.y - gb, S);
        dA += (sna + ga) - oa;
        dB += (snb + gb) - ob;
        pst(sa, sna);
        pst(sb, snb);
    }
    d.fdm[q] = make_float2(dA, dB);
    const float rt = a.x + a.y;
    const int nx = (step + 1) & 1;
    atomicAdd(&d.epend[nx * d.NT + e], make_float4(rem[0] - rt * vv.x, rem[1] - rt * vv.y, rem[2] - rt * vv.z, 0.f));
}

template <typename T>
__global__ void __launch_bounds__(128) k_fresh_apply(LbmParams p, DevState d, T* __restrict__ S, int step) {
    pdl_wait();
    pdl_trigger();
    const int nf = min(d.cnt[1], d.maxF);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += gridDim.x * blockDim.x)
        fresh_apply_node<T>(p, d, S, step, q);
}

// Owner field with the wall planes marked, empty lists, zero accumulators, correction factors 1.
__global__ void k_bb_init(LbmParams p, DevState d) {
    const unsigned int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < p.N) {
        const int z = n / p.nxy;
        d.owner[n] = wall_z(p, z) ? (uint16_t)0xFFFF : (uint16_t)0;
        d.bidx[n] = -1;
        if ((n & 31) == 0) { d.bmask[n >> 5] = 0u; d.fmask[n >> 5] = 0u; }
    }
    if (n < 2u * d.NT) {
        d.emom[n] = make_float4(0.f, 0.f, 0.f, 0.f);
        d.epend[n] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (n < (unsigned)(d.NM * d.CW * d.CW)) { d.ccnt[n] = 0; d.tcnt[n] = 0; }
    if (n < 8) d.cnt[n] = 0;
    if (n < 8) d.mass[n] = (n == 4 || n == 5) ? 1.0 : 0.0;
}

void launch_bb_init(const LbmParams& p, const DevState& d, cudaStream_t st) {
    size_t m = p.N;
    if ((size_t)2 * d.NT > m) m = (size_t)2 * d.NT;
    if ((size_t)d.NM * d.CW * d.CW > m) m = (size_t)d.NM * d.CW * d.CW;
    k_bb_init<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(p, d);
}

void launch_bb_mass(const LbmParams& p, const DevState& d, cudaStream_t st) {
    if (d.NM == 0) return;
    const double vsys = (double)p.nxy * (p.zf1 - p.zf0);
    launch_k(k_mass_finalize, dim3(1), dim3(1024), 0, st, d, vsys);
}

void launch_bb_fresh(const LbmParams& p, const DevState& d, float* Snew, int step, cudaStream_t st) {
    launch_bb_mass(p, d, st);
    launch_bb_fresh_nodes(p, d, Snew, step, st);
}

void launch_bb_fresh_nodes(const LbmParams& p, const DevState& d, float* Snew, int step, cudaStream_t st) {
    if (d.NM == 0) return;
    const size_t need_c = ((size_t)d.maxF + 7) / 8, need_a = ((size_t)d.maxF + 127) / 128;
    with_storage(p.store, [&](auto* tag) {
        using T = std::remove_pointer_t<decltype(tag)>;
        T* Sn = reinterpret_cast<T*>(Snew);
        static const int per_c = occupancy((const void*)k_fresh_compute<T>, 256);
        static const int per_a = occupancy((const void*)k_fresh_apply<T>, 128);
        launch_k(k_fresh_compute<T>, dim3(fill_grid(per_c, need_c)), dim3(256), 0, st, p, d, Sn);
        launch_k(k_fresh_apply<T>, dim3(fill_grid(per_a, need_a)), dim3(128), 0, st, p, d, Sn, step);
    });
}

}  // namespace scbb
