/*
 * scbb — two-component Shan-Chen D3Q19 lattice Boltzmann fluid coupled to triangulated soft-capsule
 * membranes, one GB300 GPU (sm_103a).  C ABI.
 *
 * Method: Wouters, Aouane, Krueger, Harting, "Mesoscale simulation of soft particles with tunable contact
 * angle in multi-component fluids" (arXiv:1904.11386).  The calls follow the paper's statement of the
 * problem: a lattice (Sec. II.A), two fluid components with a pseudo-potential coupling (Sec. II.D), a
 * relaxation time (Eq. 1), membranes with reference shapes and elastic moduli (Sec. II.B), and step(n).
 *
 * Conventions shared by every call
 *   - Units: dx = dt = rho0 = 1 (Sec. III).  Lattice node (x, y, z) has linear index x + nx*(y + ny*z);
 *     host field arrays are double[nz][ny][nx] (x fastest).
 *   - x and y are periodic.  With walls = 1 the planes z = 0 and z = nz-1 are solid wall nodes and the
 *     fluid lives on 1 <= z <= nz-2 (half-way bounce-back walls at z = 0.5 and z = nz-1.5).
 *   - Ownership: the caller owns all memory.  Device memory comes from ONE caller-allocated workspace of
 *     scbb_workspace_bytes() bytes (for example a torch uint8 CUDA tensor); the library never allocates
 *     device memory.  Host arrays passed in are copied during the call and never retained.
 *   - Streams: every kernel runs on the caller's CUDA stream given to scbb_create.  Calls that return
 *     host data synchronise that stream; scbb_step does not.
 *   - Errors: every call returns a scbb_status; nothing throws across the ABI.  scbb_last_error() gives a
 *     one-line description of the last failure on a context.  A device-side error (non-finite or
 *     non-positive density, or |u| > 0.3) is recorded in a device word and reported by the next synchronising call as
 *     SCBB_E_UNSTABLE; after it, calls other than scbb_destroy return SCBB_E_STATE.
 *   - A NULL context, NULL required pointer, or out-of-range parameter gives SCBB_E_INVAL and changes
 *     nothing.
 */
#ifndef SCBB_H
#define SCBB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCBB_ABI_VERSION 2

typedef struct scbb_ctx scbb_ctx;

typedef enum {
    SCBB_OK = 0,
    SCBB_E_INVAL = 1,        /* bad argument */
    SCBB_E_CUDA = 2,         /* a CUDA runtime call failed */
    SCBB_E_NOMEM = 3,        /* workspace smaller than scbb_workspace_bytes() */
    SCBB_E_UNSTABLE = 4,     /* non-finite density or Mach guard |u| > 0.3 tripped on the device */
    SCBB_E_TIMEOUT = 5,      /* a bounded device wait gave up */
    SCBB_E_MESH = 6,         /* invalid mesh (index out of range, zero-area reference triangle, ...) */
    SCBB_E_STATE = 7,        /* context is in an error state */
    SCBB_E_UNSUPPORTED = 8   /* a mode the library does not provide for these arguments */
} scbb_status;

/* Lattice (Sec. II.A).  walls: 1 = solid planes z=0 and z=nz-1 with half-way bounce-back (Eq. 11), 0 = periodic
 * in z.  wall_kind (with walls = 1): 0 = the walls move at u_lo / u_hi (the bounce-back's v0); 1 = the walls rest
 * and on-site velocity boundaries (Zou and He, in the D3Q19 form of Hecht and Harting, as Sec. III.A and III.C
 * impose their shear) hold the planes of fluid nodes next to them, z = 1 and z = nz-2, at u_lo and u_hi: the
 * populations those nodes receive from the wall are replaced so that each component moves at the plane's
 * velocity.  wall_kind 1 needs walls = 1 and nz >= 5 (else SCBB_E_INVAL), tau = 1 and no bounce-back membranes
 * (the fresh-node mass correction of Eq. 18 tracks the mass the lattice itself conserves; on-site planes
 * exchange mass with the outside); otherwise scbb_create returns SCBB_E_UNSUPPORTED. */
typedef struct {
    int nx, ny, nz;
    int walls;
    double u_lo[3], u_hi[3];
    int wall_kind;
} scbb_lattice;

/* Fluid (Sec. II.A, II.D, II.E).
 *   tau       BGK relaxation time (Eq. 1), > 0.5
 *   G         inter-component coupling G^{AB} = G^{BA} (Eq. 13); G^{AA} = G^{BB} = 0
 *   psi_kind  0: psi = 1 - exp(-rho) (the paper), 1: psi = rho
 *   g         uniform body acceleration; component c feels the force density rho^c g
 *   coupling  0: half-way bounce-back membranes with wetting (the paper, Sec. II.C-E),
 *             1: 2-point immersed boundary (Peskin hat; not in the paper; colour must be 0)
 *   rho_maj, rho_min   equilibrium majority / minority densities used to turn colour into a virtual
 *             density offset (Eq. 15): rho_virtual = |colour| (rho_maj - rho_min) / 2, the normalisation
 *             under which a rigid sphere's contact angle follows cos theta = colour (Sec. III.D)
 *   C0, mass_correction   adaptive fresh-node mass correction (Eq. 18), C0 = 2500 in the paper
 *   pp_eps, pp_d0         particle-particle repulsion (Eq. 26, Sec. III.E), 0.5 and 1.25 in the paper
 *   storage   0: FP32 populations; 1: populations stored as IEEE FP16, 2: as BF16 (arithmetic stays FP32;
 *             each stored value is rounded to nearest even, at most 2^-12 relative for FP16 and 2^-9 for
 *             BF16), half the population bytes; 3 / 4: the deviations f_i^c - w_i rho_ref stored as FP16 / BF16,
 *             with rho_ref = (rho_maj + rho_min) / 2 for both components (the rounding is then relative to the
 *             deviation; two-kernel bulk phase only, tau = 1).  Not in the paper.
 *   max_boundary  capacity of the bounce-back boundary-node list (nodes with a membrane-cut link); 0 sizes it
 *             from the membrane areas (three node layers per unit area, 50 % margin, + 4096).  The fresh-node
 *             list holds max_boundary / 2 + 1024.  A list that overflows keeps its first entries, skips the
 *             rest and raises the device error word: the next synchronising call returns SCBB_E_UNSTABLE.
 * 16-bit storage and the bounce-back coupling with meshes need a bulk kernel that stores every node whole: with
 * tau = 1 (the paper's value) any nx up to 256, or nx a multiple of 4 up to 2048; with tau != 1 nx a multiple of
 * 4 with nx/4 a power of two up to 32 or a multiple of 32.  Otherwise scbb_create returns SCBB_E_UNSUPPORTED. */
typedef struct {
    double tau, G;
    int psi_kind;
    double g[3];
    int coupling;
    double rho_maj, rho_min, C0;
    int mass_correction;
    double pp_eps, pp_d0;
    int storage;
    int max_boundary;
} scbb_fluid;

/* One capsule membrane (Sec. II.B): a closed triangulated surface, triangles counter-clockwise seen from
 * outside.  ref_xyz is the stress-free shape (A0 and V0 are taken from it), init_xyz the initial shape
 * (may equal ref_xyz).  kS, C: Skalak moduli (Eq. 6); kV: volume penalty (Eq. 7); kB: Helfrich bending
 * (Eq. 9-10); mass: node mass for the bounce-back coupling (5 in the paper); colour: particle colour
 * Delta rho (Eq. 15), positive prefers component A.  elem_colour: NULL, or the colour of each triangle (nt
 * values, a Janus particle; Sec. V names it as a direct extension), which then replaces colour. */
typedef struct {
    int nv, nt;
    const double* ref_xyz;   /* [nv][3] */
    const int* tri;          /* [nt][3] vertex indices 0..nv-1 */
    const double* init_xyz;  /* [nv][3] */
    double kS, C, kB, kV, mass, colour;
    const double* elem_colour;  /* [nt] or NULL */
} scbb_mesh;

/* Bytes of device workspace a context with this description needs (0 on invalid input).  The populations take
 * one lattice of 2 * 19 * N values (FP32, or 16-bit with storage 1 to 4), updated in place by the two-kernel
 * bulk phase, plus 5 N doubles of staging for the host's fields; a context with bounce-back membranes, or one
 * whose bulk phase is a fused kernel (tau != 1, or rows too long for the two-kernel phase), takes two lattices
 * (read one, write the other), the spare one staging the fields. */
size_t scbb_workspace_bytes(const scbb_lattice* lat, const scbb_fluid* fl, int n_mesh, const scbb_mesh* meshes);

/* Create a context.  dev_workspace: device pointer, 256-byte aligned, of at least `bytes` bytes, owned by
 * the caller and kept alive until scbb_destroy.  cuda_stream: a cudaStream_t (NULL = legacy default).
 * Copies the meshes to the device, precomputes reference data (reference metrics, areas, V0) and leaves
 * the fluid at rest with rho^A = rho^B = 0 until scbb_set_density.  *out receives the context. */
scbb_status scbb_create(const scbb_lattice* lat, const scbb_fluid* fl, int n_mesh, const scbb_mesh* meshes,
                        void* dev_workspace, size_t bytes, void* cuda_stream, scbb_ctx** out);

/* Initial state: populations = equilibrium (Eq. 2) of host densities rhoA, rhoB (double[N]) and host
 * velocity u (double[3][N], NULL = at rest).  Resets the vertices to init_xyz at rest.  Synchronous. */
scbb_status scbb_set_density(scbb_ctx* ctx, const double* rhoA, const double* rhoB, const double* u);

/* Advance n time steps (Eq. 1 for both components with the Shan-Chen force of Eq. 13, membrane forces of
 * Eq. 6-10, coupling, node update).  Asynchronous on the context stream.  After the context's first step,
 * pairs of steps are replayed from a CUDA graph captured on that stream (not while timing is enabled, and
 * never on the legacy default stream, where capture is not allowed: there every step launches its kernels
 * one by one; environment SCBB_GRAPHS=0 does the same everywhere).  In a context with meshes, kernels whose
 * inputs are ready early run on a second stream the context creates and joins back within the step
 * (environment SCBB_OVERLAP=0 keeps them on the context stream).  The results do not depend on either. */
scbb_status scbb_step(scbb_ctx* ctx, long long n);

/* Wait for the context stream; reports device-side errors. */
scbb_status scbb_sync(scbb_ctx* ctx);

/* Moments of the current state (post-streaming, before the next collision): rho^c = sum_i f_i^c and the
 * barycentric velocity u = sum_c sum_i f_i^c c_i / sum_c rho^c, into host double[N], double[N],
 * double[3][N] (any may be NULL).  Wall nodes report 0.  Synchronous. */
scbb_status scbb_get_fields(scbb_ctx* ctx, double* rhoA, double* rhoB, double* u);

/* Current populations f_i^c(x) (post-streaming) into host double[2][N][19] in the D3Q19 order
 * rest, +x, -x, +y, -y, +z, -z, (+x+y), (-x-y), (+x-y), (-x+y), (+x+z), (-x-z), (+x-z), (-x+z), (+y+z),
 * (-y-z), (+y-z), (-y+z).  Wall nodes report 0.  Synchronous. */
scbb_status scbb_get_populations(scbb_ctx* ctx, double* f);

/* All vertices of all meshes, concatenated in creation order: positions, velocities and the total node
 * force of the last step, host double[NV][3] each (any may be NULL).  Synchronous. */
scbb_status scbb_get_vertices(scbb_ctx* ctx, double* x, double* v, double* F);

/* FP64 reductions computed on the device: mass2[2] = total mass per component over fluid nodes, mom3[3] =
 * total fluid momentum sum_c sum_i f c, and per mesh vol[n_mesh] (enclosed volume) and com[n_mesh][3]
 * (vertex average).  Any pointer may be NULL.  Synchronous. */
scbb_status scbb_get_diag(scbb_ctx* ctx, double* mass2, double* mom3, double* vol, double* com);

/* Bounce-back coupling only: the owner of every lattice node (0 = outside all capsules, k+1 = inside mesh k,
 * 65535 = wall node) as host unsigned short[N] (may be NULL), the number of boundary nodes (nodes with a
 * link cut by a membrane, Sec. II.C) and of the fresh nodes of the last step (Sec. II.E).  Synchronous.
 * SCBB_E_UNSUPPORTED for the immersed-boundary coupling. */
scbb_status scbb_get_owner(scbb_ctx* ctx, unsigned short* owner, int* n_boundary, int* n_fresh);

/* The boundary list the next step's boundary kernel will use (built at the current positions) and the element
 * of each of its cut links (Sec. II.C): the triangle the link's segment crosses nearest to the link's node of
 * lower linear index, lower triangle id on ties; a cut link with no crossing (round-off) takes the triangle
 * of the searched capsule whose centroid is nearest the link's midpoint.  The searched capsule is the one
 * the node lies in, else the one across the link.  Writes the first min(n, max_nodes) boundary nodes (linear
 * node index, in the list's own order) to nodes[] and their elements to elems[max_nodes][18] (slot i-1 for
 * direction i of the D3Q19 order of scbb_get_populations; -1 for a link that is not cut), the list's length n
 * to *n_boundary (may be NULL; a list that overflowed its capacity holds its first maxB nodes and raises the
 * error word at the next synchronising call) and the number of cut links resolved by the nearest-centroid rule to *n_fallback (may be
 * NULL).  max_nodes = 0 with NULL arrays reads the counts alone.  Synchronous; it adds one kernel launch and
 * leaves the state as it was.  SCBB_E_INVAL for max_nodes < 0 or missing arrays, SCBB_E_UNSUPPORTED for the
 * immersed-boundary coupling. */
scbb_status scbb_get_boundary(scbb_ctx* ctx, int max_nodes, int* nodes, int* elems, int* n_boundary,
                              int* n_fallback);

/* Number of kernel launches issued by this context since creation (for launch accounting). */
long long scbb_launch_count(const scbb_ctx* ctx);

/* Measurement support.  With on = 1 or 2, every later launch of the fused bulk fluid kernel is bracketed by
 * a pair of CUDA events on the context stream (up to 4096 launches; later launches run untimed).
 * scbb_kernel_time synchronises, returns the summed device time of the timed bulk launches in
 * milliseconds and their count, and clears the record.  With on = 2 every step (up to 1024) also records
 * events between its phases; scbb_phase_times synchronises, writes the summed milliseconds of each phase
 * to ms[SCBB_PHASES] (indices below; a phase the coupling does not have reads 0) and the number of steps,
 * and clears the record.  on = 0 stops timing; other values give SCBB_E_INVAL.  Timing adds no kernel
 * launches, but the events between phases add a little time to the steps they time. */
#define SCBB_PHASES 7
enum {
    SCBB_PHASE_IBM_SPREAD = 0,   /* membrane forces and spreading (immersed boundary) */
    SCBB_PHASE_WALLS = 1,        /* wall-plane densities and ghost densities */
    SCBB_PHASE_BULK = 2,         /* fused stream + Shan-Chen + collide */
    SCBB_PHASE_BOUNDARY = 3,     /* interpolation (immersed boundary) or boundary-node collision (bounce-back) */
    SCBB_PHASE_MEMBRANE = 4,     /* bounce-back: membrane forces with the coupling and node update */
    SCBB_PHASE_CLASSIFY = 5,     /* bounce-back: owner field, boundary list and crossed elements */
    SCBB_PHASE_FRESH = 6         /* bounce-back: mass correction factors and fresh nodes */
};
scbb_status scbb_enable_timing(scbb_ctx* ctx, int on);
scbb_status scbb_kernel_time(scbb_ctx* ctx, double* ms, long long* launches);
scbb_status scbb_phase_times(scbb_ctx* ctx, double* ms, long long* steps);

/* FP64 mass and momentum of populations already on the device, for callers that cannot allocate device
 * memory: a framework that owns the device allocator and forbids side allocations, or a loop that must not
 * take cudaMalloc's implicit synchronisation or risk running out of memory mid-run.  The paper has no
 * counterpart; this is a utility of this library.
 *   dev_f   device pointer, FP32 post-streaming populations in the layout f[c][i][x + nx*(y + ny*z)] (c = 0, 1;
 *           i in the D3Q19 order of scbb_get_populations), 2*19*nx*ny*nz floats, caller-owned, read only
 *   walls   1: the planes z = 0 and z = nz-1 are wall nodes and are left out of the sums; 0: all nodes
 *   out5    host double[5]: mass of component A, mass of component B, total momentum x, y, z
 * Allocates nothing: its scratch is a fixed file-scope device array of 512 x 5 partial sums plus 5 results
 * (about 20 KB, held on every GPU that loads the library until exit).  Inputs with more than
 * SCBB_NOALLOC_MAX_NODES nodes are rejected with SCBB_E_INVAL.  Every call looks up the array's address on
 * the current device (cudaGetSymbolAddress), copies the result to the host and synchronises cuda_stream
 * (NULL = legacy default), so it must never be called on a stream under capture; dev_f must live on the
 * current device and cuda_stream belong to it.  All calls share the one scratch array
 * (every call overwrites all of it), so calls that overlap on the GPU, from several streams or threads,
 * race and must be serialised by the caller. */
#define SCBB_NOALLOC_MAX_NODES 50000000
scbb_status scbb_population_moments_noalloc(const float* dev_f, int nx, int ny, int nz, int walls, double* out5,
                                            void* cuda_stream);

/* Autotuner of the bulk kernel's block shape (not in the paper).  The row-vectorised bulk kernel can run with
 * 512 threads per CTA (one CTA per SM) or 256 (two per SM), and with z-segments of at least 6 or at least 3
 * planes; which is fastest depends on the box.  scbb_autotune times the bulk kernel of the context's current
 * state in every shape that fits the box (one untimed launch, then reps launches between CUDA events, into the
 * spare lattice, which the next step rewrites) and keeps the fastest for the context's later steps.  The
 * results of a step do not depend on the shape.  chosen (may be NULL): the shape kept, 0 .. 3, or -1 when the
 * context runs the general bulk kernel (nx not a multiple of 4), which has no shapes, or keeps one lattice
 * updated in place (every context without bounce-back membranes on the two-kernel bulk phase: a timing launch
 * would advance its state; its kernel B runs the pair form, which has one shape).  Synchronous; call it
 * between steps, not while a batch holds the context. */
scbb_status scbb_autotune(scbb_ctx* ctx, int reps, int* chosen);

/* Bound of the bulk phase's waits on its asynchronous copies (not in the paper).  The bulk kernels of a box
 * whose rows are a multiple of 4 nodes bring their inputs into shared memory by bulk asynchronous copies
 * and wait for each on an mbarrier; a wait polls at most `polls` times (default 4194304, about a second at
 * most) and then gives up: the kernel raises bit 4 of the device error word, lets its copies land and
 * returns, so the next synchronising call reports SCBB_E_TIMEOUT and later calls SCBB_E_STATE until
 * scbb_load restores a saved state.  polls = 0 gives up at the first poll that finds a copy still in
 * flight.  SCBB_E_INVAL for polls < 0.  Call it between steps, not while a batch holds the context. */
scbb_status scbb_set_wait_limit(scbb_ctx* ctx, long long polls);

/* Batches (not in the paper): step several independent contexts together, for example a sweep of boxes of
 * different sizes and parameters.  ctxs: n distinct contexts, kept alive by the caller until
 * scbb_batch_destroy; each must run on a stream of its own (not the legacy default).  cuda_stream: the
 * batch's own stream (not the legacy default, not a context's stream).  scbb_batch_step(b, n) advances
 * every context by n steps, asynchronously: the batch stream first waits for the work already queued on
 * every context stream, and afterwards every context stream waits for the batch, so single-context calls
 * before and after stay ordered.  After each context has run one step, pairs of steps of all contexts are
 * replayed from one CUDA graph with a branch per context, so small boxes run side by side on the GPU; the
 * results equal those of stepping each context alone.  Errors: SCBB_E_INVAL for bad arguments,
 * SCBB_E_STATE if a context has failed, SCBB_E_CUDA. */
typedef struct scbb_batch scbb_batch;
scbb_status scbb_batch_create(scbb_ctx* const* ctxs, int n, void* cuda_stream, scbb_batch** out);
scbb_status scbb_batch_step(scbb_batch* batch, long long n);
void scbb_batch_destroy(scbb_batch* batch);

/* Shared bulk phase of a batch (not in the paper).  When every context runs the two-kernel bulk phase (tau = 1)
 * with the same coupling mode and storage, and there are at most 64 of them, each step of the batch can run the
 * bulk phase of all boxes as ONE persistent cooperative launch on the batch stream: the stream-and-moments
 * kernel over every box's nodes, a grid barrier, then the force-and-collision kernel over every box's (tile,
 * z-segment) work items; each context's other kernels run on its own stream before and after it.  A batch does
 * so by default when none of its contexts has bounce-back membranes; with them, the per-box bookkeeping overlaps
 * other boxes' bulk phases only when each box keeps its own (a graph branch per box), which is faster.  The
 * environment variable SCBB_BATCH_PERSISTENT=1 shares the bulk phase whenever the boxes can, 0 never (read at
 * scbb_batch_create).  Results equal those of stepping each context alone, to FP32 rounding.
 * scbb_batch_shared_bulk: 1 if the batch shares the bulk phase, else 0 (also for NULL).
 * scbb_batch_set_wait_limit: the number of polls (about 0.26 us each; default 2^22, about a second) that the
 *   grid barrier's wait makes before it gives up.  A wait that gives up leaves the step incomplete and raises
 *   bit 4 of every context's device error word, which the next synchronising call on a context reports as
 *   SCBB_E_TIMEOUT (and SCBB_E_STATE afterwards, until scbb_load).  The barrier is bounded so that a launch
 *   whose blocks cannot all run at once ends with an error instead of waiting forever; a small limit forces
 *   that path.  SCBB_E_INVAL for polls < 0.  The grid barrier keeps its two counters in the first context's
 *   workspace. */
int scbb_batch_shared_bulk(const scbb_batch* batch);
scbb_status scbb_batch_set_wait_limit(scbb_batch* batch, long long polls);

/* Reverse-mode derivative of the fluid (not in the paper, which has no adjoint).  The gradient of a loss of
 * the densities after n steps, L(rho^A(T), rho^B(T)), with respect to the Shan-Chen coupling G (Eq. 13), the
 * body acceleration g and the initial densities rho^c(0), by hand-written adjoint kernels of the step:
 * BGK collision with the velocity-shift forcing (Eq. 1-5), the pseudo-potential force (Eq. 13) whose
 * stencil the adjoint applies transposed, and streaming (pull; the adjoint pushes).
 *   With walls, the adjoint includes the moving-wall bounce-back (Eq. 11) and the walls' virtual densities
 *   in the force.  Supported contexts: FP32 storage, no on-site velocity planes, and either no meshes or
 *   capsules coupled by the 2-point immersed boundary (coupling 1, Sec. II.B-C) without particle-particle
 *   repulsion; otherwise SCBB_E_UNSUPPORTED at creation.  With capsules the vertex positions are part of the
 *   state: the adjoint steps back through the interpolation of the velocity (Eq. 6-7), the explicit vertex
 *   update, the membrane forces (Skalak Eq. 8, Helfrich bending with the cotangent discretisation, volume
 *   penalty) and their spreading (Eq. 9), which carries the force into the fluid step by the velocity shift
 *   (Eq. 5).
 *   scbb_adjoint_workspace_bytes(ctx, n, K): device bytes of the adjoint's workspace for n steps with a
 *     population checkpoint every K steps: ceil(n/K) checkpoints, K + 1 lattices, K density fields and (walls)
 *     K wall planes of one segment, two adjoint lattices and 13 + 2 floats per node of scratch; with capsules
 *     also ceil(n/K) + K + 1 copies of the vertices, K copies of the membrane state of a step (12 float4 and 3
 *     float2 and a float per triangle, 4 float4 and a float2 per vertex, 4 doubles per capsule), 7 more float4
 *     per vertex and one per triangle corner for the membrane's adjoint, and 9 floats per node for the adjoint
 *     of the spread force.  0 for bad
 *     arguments.
 *   scbb_adjoint_create(ctx, n, K, dev_workspace, out): dev_workspace caller-owned, at least that many
 *     bytes, 256-byte aligned; the adjoint keeps ctx and runs on its stream.
 *   scbb_adjoint_forward(a): runs the n steps of ctx from its current state (set by scbb_set_density, an
 *     equilibrium), storing a checkpoint at steps 0, K, 2K, ...; ctx ends at step n as scbb_step(ctx, n)
 *     leaves it.
 *   scbb_adjoint_backward(a, dL_drhoA, dL_drhoB, dL_dG, dL_dg, dL_drho0A, dL_drho0B): host arrays of N
 *     doubles in, the adjoint of the final densities; out: host dL_dG (1 double), dL_dg (3 doubles) and
 *     dL_drho0A, dL_drho0B (N doubles each; either may be NULL).  Recomputes each segment of K steps from
 *     its checkpoint, then steps the adjoint backwards through it.  Synchronous.  SCBB_E_STATE before
 *     scbb_adjoint_forward.  All arithmetic is FP32 except the FP64 sums of the parameter gradients.  For a
 *     context with capsules the vertices' adjoint is zero (use scbb_adjoint_backward_capsule to seed it).
 *   scbb_adjoint_backward_capsule(a, dL_dX, dL_drhoA, dL_drhoB, dL_dmoduli, dL_dX0, dL_dG, dL_dg): the same
 *     for a context with capsules and a loss L(X(T), rho^A(T), rho^B(T)).  In: dL_dX (host, NV x 3 doubles,
 *     the vertices in the order of scbb_get_vertices), dL_drhoA and dL_drhoB (N doubles each, or NULL for a
 *     loss without the densities).  Out: dL_dmoduli (NM x 3 doubles: dL/dkS, dL/dkB, dL/dkV of each
 *     capsule, Eq. 8 and Sec. II.C), dL_dX0 (NV x 3 doubles, the initial vertex positions; NULL to skip),
 *     dL_dG, dL_dg (NULL to skip).  SCBB_E_UNSUPPORTED for a context without capsules; SCBB_E_INVAL for a
 *     NULL dL_dX or dL_dmoduli.  The initial positions' gradient holds X(0) as the membrane's reference
 *     shape fixed (a displacement of the initial positions without a change of the reference).  The
 *     vertices' positions after the backward pass are those of step n again. */
typedef struct scbb_adjoint scbb_adjoint;
size_t scbb_adjoint_workspace_bytes(const scbb_ctx* ctx, long long n_steps, int checkpoint_every);
scbb_status scbb_adjoint_create(scbb_ctx* ctx, long long n_steps, int checkpoint_every, void* dev_workspace,
                                scbb_adjoint** out);
scbb_status scbb_adjoint_forward(scbb_adjoint* a);
scbb_status scbb_adjoint_backward(scbb_adjoint* a, const double* dL_drhoA, const double* dL_drhoB, double* dL_dG,
                                  double* dL_dg, double* dL_drho0A, double* dL_drho0B);
scbb_status scbb_adjoint_backward_capsule(scbb_adjoint* a, const double* dL_dX, const double* dL_drhoA,
                                          const double* dL_drhoB, double* dL_dmoduli, double* dL_dX0,
                                          double* dL_dG, double* dL_dg);
void scbb_adjoint_destroy(scbb_adjoint* a);

/* State save and load (checkpoint and resume; not in the paper).  scbb_state_bytes: the size of a saved state,
 * a header (shape, current lattice, step count) followed by the context's whole workspace (populations,
 * densities, vertices and velocities, element accumulators, lists and counters, mass bookkeeping).
 * scbb_save copies the state into host_buf (caller-owned, at least scbb_state_bytes); synchronous.
 * scbb_load restores a state saved from a context of the same shape (lattice, walls, meshes, storage) and
 * clears a failed context's error state; SCBB_E_INVAL for a buffer of another shape.  Steps after a load
 * continue exactly as they would have from the saved state (for the bounce-back coupling up to the order of
 * float atomic additions). */
size_t scbb_state_bytes(const scbb_ctx* ctx);
scbb_status scbb_save(scbb_ctx* ctx, void* host_buf, size_t bytes);
scbb_status scbb_load(scbb_ctx* ctx, const void* host_buf, size_t bytes);

const char* scbb_last_error(const scbb_ctx* ctx);

/* Releases host-side state.  The workspace stays owned by the caller. */
void scbb_destroy(scbb_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SCBB_H */
