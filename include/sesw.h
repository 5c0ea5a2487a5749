/*
 * sesw — split-explicit shallow-water barotropic subcycle on an unstructured
 * triangular mesh, for NVIDIA GB300 (sm_103a).
 *
 * The library advances the external (barotropic) mode of an ocean model over
 * baroclinic steps. One baroclinic step of length tau is M substeps of the
 * dissipative forward-backward scheme of Banerjee et al., "Split-explicit external
 * mode solver in finite volume sea ice ocean model FESOM2" (arXiv 2311.08241),
 * Sect. 2.2, Eq. (4.10), applied to the vertically integrated system of Eq. (4.5):
 *
 *   U^{m+1} = U^m - dt [ (f/2) e_z x (U^{m+1} + U^m) + g H^m grad(eta^m) - R ]
 *   eta^{m+1} = eta^m - dt div[ (1+theta) U^{m+1} - theta U^m ],     dt = tau/M,
 *
 * with H = H0 + eta (or H0 alone when nonlinear_h = 0), the frozen forcing R of
 * Eq. (4.4), and the time-mean transport of Eq. (4.12),
 *
 *   <<U>> = (1/M) sum_{m=1..M} U^m + (theta/M)(U^M - U^0),
 *
 * which satisfies eta^M - eta^0 = -tau div <<U>> exactly (Eq. 4.11). U^0 of each
 * step is the U^M of the previous one (Sect. 2.3).
 *
 * Placement: eta on vertices, U on triangles ("elements"). The gradient of eta on a
 * triangle is that of its linear interpolant; the divergence at a vertex is the net
 * flux out of the vertex's median-dual cell divided by the cell's area
 * (A_v = sum of A_e/3 over the incident triangles). Vectors are stored in each
 * element's own planar frame (the frame of sesw_mesh.xy). The sign of the
 * pressure-gradient term is the one Eq. (4.5) fixes (the bracket of Eq. 4.10 prints
 * the opposite sign).
 *
 * Threading: a context is used by one host thread at a time. All device work is
 * issued on the stream given to sesw_create (or sesw_set_stream).
 *
 * Errors: every int-returning call returns SESW_OK (0) or a negative status; the
 * message of the last failure is available from sesw_last_error. No C++ exception
 * crosses this interface.
 */
#ifndef SESW_H
#define SESW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SESW_OK         0
#define SESW_EINVAL    -1   /* bad argument, malformed mesh, unstable parameters */
#define SESW_ECUDA     -2   /* a CUDA runtime call failed */
#define SESW_ESTATE    -3   /* call out of order (e.g. advance before mesh upload) */
#define SESW_ETIMEOUT  -4   /* a bounded device-side wait gave up */
#define SESW_EUNSTABLE -5   /* non-finite or out-of-bound elevation detected on the device */
#define SESW_ENOMEM    -6   /* device or host allocation failed */

/* Location of a caller buffer. */
#define SESW_HOST   0
#define SESW_DEVICE 1

typedef struct sesw_ctx sesw_ctx;

/* Optional device allocator. alloc returns a device pointer of at least `bytes`
 * bytes aligned to 256 B, or NULL; free releases it. `user` is passed back
 * unchanged. When both are NULL the library uses cudaMalloc/cudaFree. */
typedef void *(*sesw_alloc_fn)(size_t bytes, void *user);
typedef void (*sesw_free_fn)(void *ptr, void *user);

/* Mesh as supplied by the caller. All pointers are HOST pointers and are only read
 * during sesw_mesh_upload (the library keeps its own copies).
 *   nv, ne     number of vertices and triangles (>= 1 each)
 *   tri        [ne][3] vertex indices in [0, nv); corners counter-clockwise in the
 *              element's frame; an edge may be shared by at most two triangles,
 *              traversed in opposite directions
 *   xy         [ne][3][2] corner coordinates (m) in the element's own planar frame
 *              (periodic meshes: unwrapped per element; sphere: the plane of the
 *              flat triangle); the frame also defines the components of U and R
 *   pos        [nv][3] vertex positions used only to order the mesh along a
 *              space-filling curve (a 2-D curve when every z is 0, else 3-D);
 *              NULL keeps the caller's order
 *   depth      [nv] rest depth H0 (m), > 0; H0 on a triangle is the corner mean
 *   coriolis   [ne] Coriolis parameter f (1/s) of each triangle
 * Optional connectivity and areas. The library derives all of them from tri and xy (the
 * edges from the triangles' sides, A_e as the area of the triangle's corners in its frame,
 * A_v = sum of A_e/3 over the triangles at v, the median-dual cell of Eq. 4.10's divergence).
 * A caller that keeps its own tables may pass them; each one given is checked against the
 * derived one and a mismatch gives SESW_EINVAL naming the first bad item. NULL (or ned = 0
 * with both edge pointers NULL) means "derive". Zero-initialise the struct so that fields
 * a caller does not know of stay NULL.
 *   ned        number of edges (each side shared by one or two triangles counts once)
 *   edge_v     [ned][2] the edge's two vertices, any order
 *   edge_e     [ned][2] the triangles on either side, any order, -1 for a coast side
 *   area_v     [nv] median-dual cell areas (m^2), equal to the derived ones within 1e-12
 *              relative
 *   area_e     [ne] triangle areas (m^2), within 1e-12 relative */
typedef struct sesw_mesh {
    int32_t nv;
    int32_t ne;
    const int32_t *tri;
    const double *xy;
    const double *pos;
    const double *depth;
    const double *coriolis;
    int32_t ned;
    const int32_t *edge_v;
    const int32_t *edge_e;
    const double *area_v;
    const double *area_e;
} sesw_mesh;

/* Scheme parameters (Eq. 4.10).
 *   g            gravity (m/s^2), > 0
 *   theta        dissipation parameter, >= 0 (the paper uses 0.14)
 *   tau          baroclinic step (s), > 0; the substep is tau/M
 *   M            substeps per baroclinic step, 1..65536
 *   nonlinear_h  1: H = H0 + eta on each triangle (corner mean); 0: H = H0
 *   scheme       0: dissipative forward-backward (Eq. 4.10, "SE");
 *                1: AB3-AM4 with dissipative coefficients (Eqs. 4.7-4.8, "SESM"); levels
 *                   before the start of a subcycle are taken equal to level 0 and <<U>> is the
 *                   mean of the AB3 transports, which keeps Eq. 4.11 exact. In
 *                   SESW_MODE_PERSISTENT, patches of at most 1536 slots and 768 own vertices
 *                   keep its state on chip and larger ones stream it from L2; patches too
 *                   large for the streaming kernel's shared memory give SESW_EINVAL (upload
 *                   in SESW_MODE_GRAPH instead)
 *   flags        bit 0 (SESW_FLAG_NO_STABILITY_CHECK): accept parameters whose Courant
 *                bound exceeds the stability limit (the bound is conservative);
 *                bit 1 (SESW_FLAG_TEST_FORCE_TIMEOUT, for testing failure detection):
 *                in SESW_MODE_PERSISTENT patch 0 never publishes its halo values and each
 *                bounded wait gives up after ~1e7 cycles instead of ~1 s, so the step
 *                ends early and sesw_status reports SESW_ETIMEOUT
 *   eta_bound    |eta| above this (m) or a non-finite value sets SESW_EUNSTABLE; <= 0 means 1e4
 *   sesm_beta, sesm_delta, sesm_gamma, sesm_zeta
 *                SESM coefficients of Eq. (4.7); all zero selects beta = 0.281105 and, with
 *                chi = theta/2, gamma = 0.083 - 0.514 chi, zeta = 0.010 - 0.135 chi,
 *                delta = 2 chi + gamma + 2 zeta + 1/2 (Eqs. dp_4, dp_6)
 *   precision    arithmetic of the substeps: SESW_PRECISION_FP32 (0, the only one): eta, U and
 *                R in FP32 with the geometry rounded once from FP64, the time mean in a
 *                compensated FP32 pair (about 48 significant bits), volume and energy in FP64;
 *                any other value gives SESW_EINVAL
 *   visc_background, visc_flow
 *                barotropic viscous regularisation R_hV = div(H A grad(U/H)) of Eq.
 *                (viscosity_BT), added to the momentum forcing with its start-of-step value
 *                subtracted (Sect. 2.2): each substep uses R + R_hV(U^m, eta^m) - R_hV(U^0, eta^0).
 *                The paper fixes neither the discretisation nor A beyond "background plus a
 *                part proportional to the velocity differences across edges"; the library
 *                takes a two-point flux between neighbouring triangles across each edge of
 *                length L, H_edge (u_nb - u) A L/d with u = U/H, H_edge the mean of the two
 *                triangles' H, d the distance of their centroids in the plane unfolded across
 *                the edge, u_nb turned into the triangle's frame, and
 *                A = visc_background (m^2/s) + visc_flow (dimensionless) |u_nb - u| L.
 *                Coast edges carry no flux. Both 0 (the default) leaves the term out; it needs
 *                scheme 0 and SESW_MODE_GRAPH. The check of the stability test also bounds the
 *                viscous number dt visc_background max_e 2 sum_edges (H0_edge/H0_e)(L/d)/A_e
 *                by 1 (reported in sesw_info.visc_number). */
#define SESW_FLAG_NO_STABILITY_CHECK 1
#define SESW_FLAG_TEST_FORCE_TIMEOUT 2
#define SESW_PRECISION_FP32 0
typedef struct sesw_params {
    double g;
    double theta;
    double tau;
    int32_t M;
    int32_t nonlinear_h;
    int32_t scheme;
    int32_t flags;
    double eta_bound;
    double sesm_beta;
    double sesm_delta;
    double sesm_gamma;
    double sesm_zeta;
    double visc_background;
    double visc_flow;
    int32_t precision;
    int32_t reserved;        /* 0 */
} sesw_params;

/* Read-only facts about the uploaded mesh and its device layout. */
typedef struct sesw_info {
    int32_t nv, ne;
    int32_t npatch;          /* vertex patches (one CTA each) */
    int32_t nslot;           /* element slots: ne owned + guest copies on patch borders */
    int32_t max_patch_slots; /* largest slot count of one patch */
    int32_t patch_vertices;  /* target vertices per patch */
    int32_t block_threads;   /* threads per block of the substep (or persistent) kernel */
    int32_t mode;            /* SESW_MODE_GRAPH or SESW_MODE_PERSISTENT (0 from sesw_mesh_check) */
    int32_t blocks_per_sm;   /* persistent mode: resident blocks per SM */
    int32_t slots_per_thread;/* persistent mode: element slots per thread (held in registers,
                                or slot-loop rounds when streamed) */
    int32_t cached;          /* persistent mode, register kernels: 1 when the static slot data lives in
                                shared memory, 2 when the vertices' data and the low parts of the
                                compensated sums do and the static slot data are read from L2
                                (large patches); streaming kernels (streamed != 0): 1 when the
                                vertices' data lives in shared memory */
    int32_t nbasin;          /* meshes in the uploaded batch (1 for sesw_mesh_upload) */
    double courant_max;      /* estimated largest substep Courant number sqrt(gH kappa^2) dt
                                (0 until parameters are set) */
    double courant_limit;    /* 2/sqrt(1+2 theta), the stability limit of the scheme */
    double stiffness_bound;  /* upper bound L (1/m) of lambda_max(-div H0 grad);
                                courant_max = (tau/M) sqrt(g L) */
    int64_t device_bytes;    /* device memory held by the context */
    int32_t npack;           /* persistent mode: cooperative launches per step (packs of meshes
                                that together fit the resident grid) */
    int32_t streamed;        /* persistent mode: nonzero when the (first) pack streams its transport,
                                sums and static slot data from L2, for patches too large for
                                registers: 1 with the slots' corner indices held in shared memory,
                                2 with them read from L2 too (the largest patches) */
    double visc_number;      /* viscous number of the barotropic viscosity (see sesw_params;
                                0 until parameters are set) */
    double visc_stiffness;   /* max_e 2 sum_edges (H0_edge/H0_e)(L/d)/A_e (1/m^2): visc_number =
                                (tau/M) visc_background visc_stiffness */
    int32_t step_graph;      /* 1 when a baroclinic step is enqueued as one CUDA graph launch (all of its
                                kernels); 0 when the cooperative launches could not be captured and are
                                issued directly */
    int32_t launches;        /* kernel launches of one step: persistent SE, one per group of packs that
                                run the same kernel (a launch runs its packs one after another);
                                persistent SESM, one per pack; graph mode, M + 1 (SE) */
} sesw_info;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). alloc/free: see sesw_alloc_fn.
 * On success *out owns the context until sesw_destroy. */
int sesw_create(sesw_ctx **out, int device, void *cuda_stream,
                sesw_alloc_fn alloc, sesw_free_fn free_fn, void *user);

/* Replace the stream used for subsequent work. */
int sesw_set_stream(sesw_ctx *ctx, void *cuda_stream);

/* Set the target number of vertices per patch (>= 32) of SESW_MODE_GRAPH for the
 * next mesh upload; default 256. (SESW_MODE_PERSISTENT sizes its patches itself so that
 * the largest mesh fills the grid of resident blocks.) */
int sesw_set_patch_vertices(sesw_ctx *ctx, int32_t patch_vertices);

/* Execution modes of a baroclinic step.
 *   SESW_MODE_GRAPH       M launches of the substep kernel (one block per patch of
 *                         ~patch_vertices vertices) plus an epilogue, as one CUDA graph
 *   SESW_MODE_PERSISTENT  one cooperative launch per step (per pack of a batch): each
 *                         block keeps its patch's elevation and fluxes in shared memory
 *                         and its transports in registers for all M substeps (patches
 *                         too large for that stream their transports and static data
 *                         from L2 instead, see sesw_info.streamed), exchanging boundary
 *                         elevation with neighbouring blocks as tagged words through L2
 *                         with bounded waits (a wait that gives up sets SESW_ETIMEOUT)
 *   SESW_MODE_AUTO        persistent when the mesh fits it, else graph (default)
 * Both modes, every patch size and every batch give bitwise the same results for the SE
 * scheme: each triangle's update is one fixed sequence of FP32 roundings, and each vertex
 * adds its incident triangles' contributions in the order of the caller's triangle ids.
 * Takes effect at the next mesh upload. */
#define SESW_MODE_AUTO       0
#define SESW_MODE_GRAPH      1
#define SESW_MODE_PERSISTENT 2
int sesw_set_mode(sesw_ctx *ctx, int32_t mode);

/* Persistent mode: which kernel form each pack (one cooperative launch) runs.
 *   SESW_FORM_AUTO             the register form where a thread holds at most 6 slots, or 7 or
 *                              8 with the vertices' data and compensation terms in shared
 *                              memory; else the streaming form (default)
 *   SESW_FORM_REGISTERS        transports and sums in registers, static slot data in shared
 *                              memory when it fits, else the vertices' data and the low parts of
 *                              the compensated sums (sesw_info.streamed = 0)
 *   SESW_FORM_STREAM           transports, sums and static data read from L2 slot by slot,
 *                              corner indices in shared memory when they fit (streamed = 1, else 2)
 *   SESW_FORM_STREAM_UNCACHED  the streaming form with the corner indices read from L2 too
 *                              (streamed = 2)
 * All forms give bitwise the same results (the per-vertex sums run in a fixed order). A mesh
 * that does not fit the requested form falls back to graph mode (SESW_MODE_AUTO) or is refused
 * (SESW_MODE_PERSISTENT). Takes effect at the next mesh upload. */
#define SESW_FORM_AUTO            0
#define SESW_FORM_REGISTERS       1
#define SESW_FORM_STREAM          2
#define SESW_FORM_STREAM_UNCACHED 3
int sesw_set_persistent_form(sesw_ctx *ctx, int32_t form);

/* Persistent mode, batches: the residency and kernel form of the packs of "large" basins,
 * those too large for one grid of patches of the common size (the largest patch whose static
 * data fits shared memory at the batch's blocks per SM, 1280 vertices at one block per SM).
 * Such a basin fills its own grid of blocks_per_sm x SMs patches; blocks_per_sm 0 (default)
 * takes the batch's own value, and form -1 (default) the form of sesw_set_persistent_form.
 * With two blocks per SM and the streaming form, for example, a 400k-vertex basin runs 304
 * patches of ~1300 vertices streamed from L2 while the small basins of the same batch keep one
 * block per SM and their static data in shared memory. Results do not depend on this choice
 * (bitwise). Takes effect at the next mesh upload. */
int sesw_set_large_basins(sesw_ctx *ctx, int32_t blocks_per_sm, int32_t form);

/* Persistent mode: resident blocks (patches) per SM, 1 to 4; 0 (default) tries 2
 * and falls back to 1. With 0, a single mesh whose patches at 2 blocks per SM do not keep all
 * their data on chip takes 1 block per SM when every patch then runs the register kernel (the
 * choice is made for the SE scheme: the SESM streaming kernel on such a mesh, e.g. the level-8
 * sphere, is faster at 2). Takes effect at the next mesh upload. */
int sesw_set_blocks_per_sm(sesw_ctx *ctx, int32_t blocks_per_sm);

/* Threads per block of the substep kernel (a multiple of 32 in [32, 1024]);
 * default 256. Takes effect at the next advance. */
int sesw_set_block_threads(sesw_ctx *ctx, int32_t threads);

/* Validate, reorder and upload a mesh (mesh prep: geometry, space-filling-curve
 * order, vertex patches with their boundary element copies, per-vertex incidence).
 * Resets state and forcing to zero. Synchronises with the device.
 * Errors: SESW_EINVAL (with a message naming the first bad item), SESW_ENOMEM,
 * SESW_ECUDA. */
int sesw_mesh_upload(sesw_ctx *ctx, const sesw_mesh *mesh);

/* Upload a batch of independent meshes ("basins", e.g. ensemble members of uneven
 * size) that advance together in every sesw_advance. Each mesh is validated and
 * prepared exactly as sesw_mesh_upload would prepare it alone (its own space-filling
 * curve order and patches), and the layouts are concatenated; a basin's results are
 * bitwise those of its own upload in any mode and layout. In SESW_MODE_PERSISTENT each basin
 * gets the larger of its one-grid patch size and a common size whose static data fits shared
 * memory (basins larger than one grid of those are cut by sesw_set_large_basins); the meshes
 * are packed, largest first, into packs that each fill at most one grid of resident blocks,
 * a step runs one cooperative launch per pack, and the launches of a step are one CUDA graph.
 * Caller order of every state,
 * forcing and output array is the concatenation of the meshes in order. Errors name
 * the first bad basin. */
int sesw_mesh_upload_batch(sesw_ctx *ctx, int32_t nmesh, const sesw_mesh *meshes);

/* Parameters of a batch, one set per mesh (n = number of uploaded meshes). All sets
 * must agree in g, theta, M, nonlinear_h, scheme, flags, eta_bound, the SESM and the
 * viscosity coefficients; tau (hence the
 * substep dt = tau/M) may differ per mesh. Each mesh gets its own stability check. */
int sesw_set_params_batch(sesw_ctx *ctx, int32_t n, const sesw_params *params);

/* Set scheme parameters; requires an uploaded mesh. Rejects (SESW_EINVAL)
 * parameters whose substep Courant number bound exceeds 2/sqrt(1+2 theta), the
 * value beyond which the scheme's characteristic polynomial (Eq. dp_1, SE row) has a
 * root outside the unit circle (for SESM the limit of its coefficients, found
 * numerically from the spectral radius of the per-mode substep matrix). c is an upper bound of dt sqrt(lambda_max(-div g H0
 * grad)) for the lumped median-dual operator: the smaller of an element-by-element
 * bound, dt sqrt(3 g max_e H0_e lambda_max(sum_k grad phi_k grad phi_k^T)), and the
 * Gershgorin bound over the rows of the stiffness matrix divided by A_v. */
int sesw_set_params(sesw_ctx *ctx, const sesw_params *params);

/* Set the state: eta [nv] (m) and U [ne][2] (m^2/s), in the caller's vertex and
 * element order, as doubles at `where` (SESW_HOST or SESW_DEVICE). U is the U^0 of
 * the next baroclinic step. Host buffers may be pageable or pinned. */
int sesw_set_state(sesw_ctx *ctx, const double *eta, const double *U, int where);

/* Set the frozen forcing R [ne][2] (m^2/s^2) of Eq. (4.4), caller order. */
int sesw_set_forcing(sesw_ctx *ctx, const double *R, int where);

/* Set the freshwater flux W [nv] (m/s, positive out of the ocean) of Eq. (4.5), caller
 * order, frozen like R: every substep then updates eta^{m+1} = eta^m - dt (div F + W),
 * so a step changes the volume by -tau sum_v A_v W_v and Eq. (4.11) reads
 * eta^{n+1} = eta^n - tau (div <<U>> + W). W = NULL removes the term (the default). All
 * schemes and modes. */
int sesw_set_freshwater(sesw_ctx *ctx, const double *W, int where);

/* Evaluate the barotropic viscous regularisation R_hV (see sesw_params) at the current
 * state with the current parameters into out [ne][2] (m^2/s^2, element frames, caller
 * order); zero when both coefficients are 0. SESW_MODE_GRAPH only. With SESW_HOST the
 * call synchronises. */
int sesw_viscosity(sesw_ctx *ctx, double *out, int where);

/* Advance nsteps >= 0 baroclinic steps (nsteps*M substeps). Asynchronous on the
 * context's stream; device-side instability is reported by sesw_status or
 * sesw_get_state. Requires mesh and parameters. */
int sesw_advance(sesw_ctx *ctx, int32_t nsteps);

/* Copy out the state in caller order as doubles: eta [nv], U = U^M [ne][2] and
 * Umean = <<U>> of the last step [ne][2] (Eq. 4.12; zero before the first step).
 * Any pointer may be NULL. With SESW_HOST the call synchronises with the stream and
 * returns SESW_EUNSTABLE if the device flagged instability; with SESW_DEVICE the
 * copies are only enqueued. */
int sesw_get_state(sesw_ctx *ctx, double *eta, double *U, double *Umean, int where);

/* Asynchronous host transfers, for callers that pipeline steps: the copies run on the
 * library's own copy streams and overlap the steps before and after them; a ticket names
 * each state read-back. Host buffers should be pinned (page-locked) for the copies to be
 * asynchronous.
 *   sesw_set_forcing_async  as sesw_set_forcing with a host R; R may be changed again once
 *                           sesw_wait has returned for a ticket issued after this call
 *   sesw_get_state_async    as sesw_get_state into host buffers (any may be NULL); returns
 *                           at once with *ticket > 0; the buffers hold the state once
 *                           sesw_wait(ctx, ticket) returns
 *   sesw_wait               waits until the read-back `ticket` has landed (0: until every
 *                           transfer and step issued so far has finished); returns
 *                           SESW_EUNSTABLE if the device had flagged instability by then,
 *                           SESW_EINVAL for a ticket not issued yet. */
int sesw_set_forcing_async(sesw_ctx *ctx, const double *R);
int sesw_get_state_async(sesw_ctx *ctx, double *eta, double *U, double *Umean, uint64_t *ticket);
int sesw_wait(sesw_ctx *ctx, uint64_t ticket);

/* Keep (enable = 1) or stop keeping (0) the step-mean elevation
 * eta_bar = (1/M) sum_{m=0..M-1} eta^m of every baroclinic step (SE scheme): the time
 * mean that enters the exactly summed momentum equation of a step,
 * U^M - U^0 + tau [ f e_z x S' + g H grad(eta_bar) - R ] = 0 (linear H), with
 * S' = <<U>> - (theta/M)(U^M - U^0) + (U^0 - U^M)/(2M). Costs one read-modify-write per
 * vertex and substep while enabled. */
int sesw_set_eta_mean(sesw_ctx *ctx, int32_t enable);

/* Copy out eta_bar of the last step [nv] in caller order (host: synchronises). */
int sesw_get_eta_mean(sesw_ctx *ctx, double *eta_mean, int where);

/* FP64 diagnostics of the current state: volume sum_v A_v eta_v (m^3) and energy
 * sum_v A_v g eta_v^2/2 + sum_e A_e |U_e|^2 / (2 H_e) (m^5/s^2). Synchronises. */
int sesw_diagnostics(sesw_ctx *ctx, double *volume, double *energy);

/* Per-mesh FP64 diagnostics of a batch: volume[b] and energy[b] for every uploaded
 * mesh b (arrays of nbasin host doubles). Synchronises. */
int sesw_diagnostics_batch(sesw_ctx *ctx, double *volume, double *energy);

/* Allocation-free volume and energy of a caller-held state. The paper has no
 * counterpart: this serves callers that cannot allocate device memory where they need
 * the numbers (code running inside another framework's memory pool or under its
 * allocator lock, loops that must not enter the CUDA allocator, hosts that only hand
 * over pre-allocated buffers). It needs no context and computes
 *   out[0] = sum_v area_v[v] eta[v]
 *   out[1] = sum_v area_v[v] g eta[v]^2 / 2 + sum_e area_e[e] |U[e]|^2 / (2 h_e[e]),
 * the quantities of sesw_diagnostics, in FP64.
 * Arguments: device pointers on the current device, caller order and caller-owned:
 * area_v and eta [nv], area_e and h_e (water depth H of each triangle, > 0) [ne],
 * U [ne][2], out [2]; g > 0; cuda_stream a cudaStream_t (NULL = legacy default).
 * Work is enqueued on the stream and the call returns without waiting.
 * Limits: 0 <= nv, ne <= SESW_NOALLOC_MAX_ITEMS (33,554,432); larger sizes, NULL
 * pointers and a g that is not positive return SESW_EINVAL before anything is launched
 * (the device data, such as h_e > 0, is not checked); a failed launch returns SESW_ECUDA.
 * Scratch: one fixed 128 KiB array of partial sums (SESW_NOALLOC_MAX_CHUNKS pairs of
 * doubles) that lives in the library's device memory on every GPU that loads the
 * library, until the process exits. Nothing is allocated or freed by the call. Every
 * call reuses the same array and overwrites the partials it needs (nothing has to
 * start at zero); calls that overlap on the GPU (several streams or threads at once)
 * race on it and must be ordered by the caller.
 * The first call on a device looks up the array's device address with that device
 * current (cudaGetSymbolAddress) and keeps it for the rest of the process; make that first
 * call before any stream capture, and do not call this after a cudaDeviceReset of the
 * device in the same process (the kept address would be stale). */
#define SESW_NOALLOC_MAX_CHUNKS 8192
#define SESW_NOALLOC_MAX_ITEMS (SESW_NOALLOC_MAX_CHUNKS * 4096)
int sesw_diagnostics_noalloc(int64_t nv, int64_t ne, const double *area_v, const double *eta,
                             const double *area_e, const double *h_e, const double *U, double g,
                             double *out, void *cuda_stream);

/* ---- Learned surrogate of one baroclinic step (SE scheme, single mesh).
 * The paper has no surrogate. A message-passing network (3 layers, width 64, bfloat16
 * weights, float accumulation; vertex inputs eta/s_eta and H0/s_H; element inputs U/s_U,
 * R/s_R, f/s_f and H0_e/s_H; each layer updates elements from the P1 gradients of the
 * vertex features and vertices from the area-weighted mean of the element features)
 * predicts the increments of <<U>> (Eq. 4.12), of U^M and of the step-mean elevation
 * eta_bar over one step. Its kernels (forward, backward, Adam) run on the context's
 * stream. Scales s = (eta, H, U, R, f, L, out_U, out_eta): L multiplies the P1 gradients;
 * out_U and out_eta scale the two output groups. Samples live on the device in the
 * library's order; inputs in caller order are converted on the way in. */

/* Create the surrogate for the uploaded mesh with room for `capacity` samples;
 * weights Glorot-uniform from `seed`, scales 1. Replaces an existing surrogate. */
int sesw_surrogate_init(sesw_ctx *ctx, int32_t capacity, int32_t seed);
/* Number of parameters (floats). */
int sesw_surrogate_nparam(sesw_ctx *ctx, int64_t *nparam);
/* Read (get != NULL) and/or replace (set != NULL) the float master weights [nparam], host. */
int sesw_surrogate_weights(sesw_ctx *ctx, float *get, const float *set);
/* Read (get) and/or replace (set) the 8 scales, host doubles; scales must be > 0. */
int sesw_surrogate_scales(sesw_ctx *ctx, double *get, const double *set);
/* Store sample `index`: inputs eta [nv], U [ne][2], R [ne][2] and targets
 * <<U>> - U [ne][2], U^M - U [ne][2], eta_bar - eta [nv], caller order, doubles at `where`. */
int sesw_surrogate_set_sample(sesw_ctx *ctx, int64_t index, const double *eta, const double *U,
                              const double *R, const double *d_umean, const double *d_um,
                              const double *d_etabar, int where);
/* Store the context's current state and forcing as the inputs of sample `index`
 * (call before sesw_advance(ctx, 1)) ... */
int sesw_surrogate_record_input(sesw_ctx *ctx, int64_t index);
/* ... and the result of that step as its targets (needs sesw_set_eta_mean(ctx, 1)). */
int sesw_surrogate_record_target(sesw_ctx *ctx, int64_t index);
/* Set the scales from the RMS of samples [0, nsamples) (eta, U, R, both output groups),
 * the largest |H0_e| and |f|, and length_scale for L. */
int sesw_surrogate_fit_scales(sesw_ctx *ctx, int64_t nsamples, double length_scale);
/* One Adam step (learning_rate, betas 0.9/0.999, eps 1e-8) per listed sample, in order;
 * mean_loss (may be NULL) receives the mean of the losses before each step. The loss
 * is the mean squared error of the normalised outputs over elements and channels plus
 * that over vertices. */
int sesw_surrogate_train(sesw_ctx *ctx, const int64_t *indices, int32_t n, double learning_rate,
                         double *mean_loss);
/* Mean loss of the listed samples without training. */
int sesw_surrogate_loss(sesw_ctx *ctx, const int64_t *indices, int32_t n, double *mean_loss);
/* Loss of sample `index` and its gradient with respect to the weights [nparam] (host). */
int sesw_surrogate_gradient(sesw_ctx *ctx, int64_t index, float *grad, double *loss);
/* Normalised outputs for sample `index`, caller order: out_e [ne][4], out_v [nv] (host). */
int sesw_surrogate_predict(sesw_ctx *ctx, int64_t index, double *out_e, double *out_v);
/* Advance nsteps steps with the surrogate. Each step applies the predicted <<U>> and U^M,
 * sets eta^{n+1} = eta^n - tau div <<U>> (exact volume, Eq. 4.11 holds), and measures the
 * residual of the step's exactly summed momentum equation,
 *   r = U^M - U^0 + tau [ f e_z x S' + g H grad(eta_bar) - R ],
 *   S' = <<U>> - (theta/M)(U^M - U^0) + (U^0 - U^M)/(2M),
 * as sqrt(sum A |r|^2 / sum A |U^M - U^0|^2). A step whose residual exceeds resid_tol is
 * undone and taken by the plain subcycle; *n_fallback counts those steps and
 * *last_resid receives the last residual (either may be NULL). Synchronises per step.
 * Refused (SESW_EINVAL) while the barotropic viscosity or a freshwater flux is set: the
 * network and the residual check know neither term. */
int sesw_surrogate_advance(sesw_ctx *ctx, int32_t nsteps, double resid_tol, int32_t *n_fallback,
                           double *last_resid);

/* Synchronise and return SESW_OK, SESW_EUNSTABLE or SESW_ETIMEOUT from the device
 * status word; clears the word. */
int sesw_status(sesw_ctx *ctx);

/* Validate and lay out a mesh on the host only, with no device involved: the
 * checks and the patch layout of sesw_mesh_upload for `patch_vertices` vertices per
 * patch. On success fills info (courant fields and device_bytes 0). On failure
 * returns SESW_EINVAL and copies the message into msg (NUL-terminated, at most
 * msglen bytes; msg may be NULL). */
int sesw_mesh_check(const sesw_mesh *mesh, int32_t patch_vertices, sesw_info *info,
                    char *msg, size_t msglen);

/* Mesh and layout facts; requires an uploaded mesh. */
int sesw_get_info(sesw_ctx *ctx, sesw_info *info);

/* Message of the last failed call on this context ("" if none). Valid until the
 * next call on the context. */
const char *sesw_last_error(sesw_ctx *ctx);

/* Release all device and host resources. NULL is ignored. */
void sesw_destroy(sesw_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SESW_H */
