// Internal declarations shared by the host side (mesh prep, C-ABI) and the CUDA
// kernels of libsesw. Not part of the public interface (include/sesw.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sesw.h"

namespace sesw {

// Mesh after preparation, in the library's order.
//
// Vertices are sorted along a Hilbert curve and cut into contiguous patches; each
// patch is processed by one thread block. An element is owned by the patch of its
// lowest-numbered corner; a patch also holds a "guest" copy of every element owned
// elsewhere that touches one of its vertices, so the vertex update of a patch only
// needs element results computed inside the same block. Guest copies evolve with
// the same instructions on the same inputs as the owner copy and so stay bitwise
// identical to it.
//
// Slot s (0 <= s < nslot) is one element copy. Patch p holds slots
// [patch_slot[p], patch_slot[p+1]); its first patch_own[p] slots are the elements it
// owns, in element order, then its guests.
struct HostMesh {
    int nv = 0, ne = 0, npatch = 0, nslot = 0, max_patch_slots = 0, patch_vertices = 0;
    int max_patch_vertices = 0;
    std::vector<int> vperm;        // new vertex -> caller vertex
    std::vector<int> eperm;        // new element -> caller element
    std::vector<int> patch_v;      // [npatch+1] vertex ranges
    std::vector<int> patch_slot;   // [npatch+1] slot ranges
    std::vector<int> patch_own;    // [npatch] number of owned slots
    std::vector<int> patch_int;    // [npatch] number of interior slots (the first ones)
    std::vector<int4> slot_v;      // corners (new vertex ids); .w = element id, or -1-element for guests
    std::vector<float4> slot_g;    // (dphi0/dx, dphi0/dy, dphi1/dx, dphi1/dy); dphi2 = -dphi0 - dphi1
    std::vector<float4> slot_c;    // (A_e, H0_e, f_e, 0)
    std::vector<int> vcsr_off;     // [nv+1] incidence list of each vertex
    std::vector<uint32_t> vcsr;    // (local slot << 2) | corner, local to the vertex's patch
    std::vector<float> inv_av;     // 1 / median-dual area
    std::vector<float> h0_v;       // rest depth at vertices (new order)
    std::vector<double> area_v;    // median-dual area (FP64, for diagnostics)
    std::vector<double> area_e;    // element area (FP64), new element order
    std::vector<double> h0_e;      // element rest depth (FP64), new element order
    double grad_gram_max_h = 0.0;  // upper bound of lambda_max(-div H0 grad) (m/s^2 units without g)
    // Barotropic viscosity (Eq. viscosity_BT), new element order: neighbours across the
    // edges (corner k, corner k+1) as element ids (-1: coast), the neighbour's corner
    // opposite the edge (new vertex id), and per edge the rotation from the neighbour's
    // frame (cos, sin), L/d and L^2/d of the two-point flux.
    std::vector<int4> visc_nb;
    std::vector<int4> visc_opp;
    std::vector<float4> visc_geo;  // [ne][3]
    bool visc_rot = false;         // some neighbour frame is turned (sphere)
    double visc_stiffness = 0.0;   // max_e 2 sum_k (H0_edge / H0_e)(L/d) / A_e (1/m^2)

    // Batches: a layout may hold several independent meshes ("basins"), each prepared
    // on its own and concatenated; patches never straddle basins.
    int nbasin = 1;
    std::vector<int> patch_basin;      // [npatch]
    std::vector<int> basin_v;          // [nbasin+1] caller vertex ranges
    std::vector<int> basin_e;          // [nbasin+1] caller element ranges
    std::vector<int> basin_patch;      // [nbasin+1] patch ranges
    std::vector<double> basin_stiffness;   // per basin, as grad_gram_max_h
    std::vector<double> basin_visc_stiffness;   // per basin, as visc_stiffness

    // Halo structure for the persistent kernel (filled by build_halos). A patch keeps
    // its own vertices at local indices [0, n_own) and its halo vertices (corners of
    // its slots owned by other patches) at [n_own, n_own + n_halo).
    std::vector<int> patch_halo;   // [npatch+1] ranges into halo_v
    std::vector<int> halo_v;       // halo vertex ids (new order), sorted per patch
    std::vector<ushort4> slot_l;   // local corner indices of each slot (.w unused)
    int max_patch_local = 0;       // max n_own + n_halo
    int max_patch_halo = 0;        // max n_halo
    int max_patch_csr = 0;         // max incidence entries of one patch's own vertices
};

// Concatenate independently prepared meshes (each with patch_basin all 0) into one
// layout; caller order of the result is the concatenation of the inputs' caller orders.
void concat_meshes(std::vector<HostMesh> &parts, HostMesh &out);

// Fill the halo structure of a prepared mesh. Returns SESW_OK or SESW_EINVAL when a
// patch needs local indices beyond 16 bits.
int build_halos(HostMesh &hm, std::string &err);

// Validate and prepare; returns SESW_OK or SESW_EINVAL with a message in err.
int prepare_mesh(const sesw_mesh &m, int patch_vertices, HostMesh &out, std::string &err);

// Hilbert keys (exposed for tests of the ordering).
uint64_t hilbert2d(uint32_t x, uint32_t y, int bits);
uint64_t hilbert3d(uint32_t x, uint32_t y, uint32_t z, int bits);

// Device arrays of one prepared mesh plus the state.
struct DevMesh {
    int nv = 0, ne = 0, npatch = 0, nslot = 0, max_patch_slots = 0;
    int4 *slot_v = nullptr;
    float4 *slot_g = nullptr;
    float4 *slot_c = nullptr;
    int *patch_v = nullptr;
    int *patch_slot = nullptr;
    int *patch_own = nullptr;
    int *patch_int = nullptr;
    int *vcsr_off = nullptr;
    uint32_t *vcsr = nullptr;
    float *inv_av = nullptr;
    float *h0_v = nullptr;
    double *area_v = nullptr;
    double *area_e = nullptr;      // FP64 element area and rest depth (new element order), for the
    double *h0_e = nullptr;        // FP64 diagnostics
    int *vperm = nullptr;
    int *eperm = nullptr;
    // caller-order maps of the state transfers
    int *slot_e = nullptr;         // [nslot] caller element of each slot (owner and guest copies)
    int *einv = nullptr;           // [ne] caller element -> new element
    int *eown = nullptr;           // [ne] caller element -> its owner slot
    int *vinv = nullptr;           // [nv] caller vertex -> new vertex
    float *patch_dt = nullptr;     // [npatch] substep length tau/M of the patch's basin
    float4 *slot_k = nullptr;      // [nslot] the persistent kernels' step coefficients of each slot,
                                   // (dt A_e, g H0_e, f dt / 2, 1 / (1 + (f dt / 2)^2)), set with the parameters
    // barotropic viscosity, per slot (graph mode): edge k joins corners k and k+1; q_k is
    // the neighbour's owner slot (-1: coast), c_k its corner opposite the edge, h_k its
    // H0, a_k = L/d, b_k = L^2/d, (cos, sin)_k the turn from its frame into this one
    int4 *visc_q = nullptr;        // (q0, q1, q2, bits of h0)
    int4 *visc_c = nullptr;        // (c0, c1, c2, bits of h1)
    float4 *visc_a = nullptr;      // (a0, a1, a2, h2)
    float4 *visc_b = nullptr;      // (b0, b1, b2, 0)
    float4 *visc_r = nullptr;      // (cos0, sin0, cos1, sin1), only when visc_rot
    float2 *visc_r2 = nullptr;     // (cos2, sin2), only when visc_rot
    int visc_rot = 0;
    int nbasin = 1;
    int *basin_v = nullptr;        // [nbasin+1] vertex ranges (new order = caller order per basin)
    int *basin_slot = nullptr;     // [nbasin+1] slot ranges
    // persistent mode: patches grouped into packs that each fit the resident grid; a
    // step launches the packs one after another
    int *pack_patch = nullptr;     // [npatch] patch ids, pack by pack
    std::vector<int> pack_off;     // [npack+1] ranges into pack_patch (host)
    int *pack_off_d = nullptr;     // the same on the device
    // persistent kernel
    int *patch_halo = nullptr;
    int *halo_v = nullptr;
    ushort4 *slot_l = nullptr;
    int max_patch_local = 0, max_patch_vertices = 0, max_patch_halo = 0, max_patch_csr = 0;
};

struct DevState {
    float *eta[2] = {nullptr, nullptr};   // ping-pong elevation, new vertex order
    float2 *U = nullptr;                  // per slot
    float2 *R = nullptr;                  // per slot
    float2 *S_hi = nullptr;               // per slot, compensated running sum of the substep fluxes
    float2 *S_lo = nullptr;
    float2 *Umean = nullptr;              // per new element
    unsigned *status = nullptr;           // device status word (bit 0: unstable, bit 1: timeout)
    double *diag_part = nullptr;          // per-block partial sums of the diagnostics
    double *diag_out = nullptr;           // [2] volume, energy
    double *stage = nullptr;              // FP64 staging for host/device transfers
    size_t stage_elems = 0;
    // persistent kernel
    float *xbuf[2] = {nullptr, nullptr};  // boundary elevation exchanged between patches, per substep parity
                                          // (persistent kernel: 64-bit tagged words, 2 floats per vertex)
    unsigned *flags = nullptr;            // substeps completed by each patch in the running step, one
                                          // 128-byte line per patch, then the abort word
    unsigned *abort_flag = nullptr;       // set by a block whose bounded wait gave up
    // SESM (graph mode): five elevation levels (eta[0], eta[1] and three more) and two
    // extra transport levels per slot (U is the third)
    float *eta_x[3] = {nullptr, nullptr, nullptr};
    float2 *U_x[2] = {nullptr, nullptr};
    // optional sum of eta^0 .. eta^{M-1} over the last step (SE; cleared at each step start)
    float *eta_sum = nullptr;
    // freshwater flux W (m/s, positive out of the ocean), new vertex order; NULL when unset
    float *W = nullptr;
    // barotropic viscosity (SE, graph mode): its start-of-step value per slot
    float2 *V0 = nullptr;
};

// Viscosity coefficients of one launch (Eq. viscosity_BT): A = background + flow |du| L.
struct ViscArgs {
    float background, flow;
    int nonlinear_h;
};

// A substep with the barotropic viscosity (graph mode): transports are read from U_in
// (U^m) and written to U_out (U^{m+1}); start = 1 on substep 0 of a step, which stores
// the term's start-of-step value in DevState::V0.
struct SubstepViscArgs {
    ViscArgs va;
    int start;
    const float2 *U_in;
    float2 *U_out;
};

// Level pointers of one SESM launch (see k_sesm).
struct SesmPtrs {
    const float2 *u1, *u2, *u3;
    float2 *u0;
    const float *e0, *e1, *e2, *e3;
    float *enew;
    int update, vertex;
};

// Scheme constants shared by all patches (the substep dt is per patch, DevMesh::patch_dt).
struct StepArgs {
    float g, theta, inv_M, eta_bound;
    float ab0, ab1, ab2;            // SESM: AB3 weights (Eq. 4.7)
    float am0, am1, am2, am3;       // SESM: AM4 weights (Eq. 4.7)
    int nonlinear_h;
    int silent_patch;          // persistent kernel: this patch never publishes its halo values (-1: none; test hook)
    long long wait_cycles;     // persistent kernel: budget of one bounded wait, in SM clock cycles
    double g64;
};

// Kernel launchers (sesw_kernels.cu). All enqueue on `stream` and return the
// launch error.
cudaError_t launch_substep(const DevMesh &m, const DevState &s, const StepArgs &a, int parity,
                           int block, cudaStream_t stream, const SubstepViscArgs *visc = nullptr);
cudaError_t substep_smem_attr(const DevMesh &m);
cudaError_t launch_step_epilogue(const DevMesh &m, const DevState &s, const StepArgs &a,
                                 cudaStream_t stream);
cudaError_t launch_sesm(const DevMesh &m, const DevState &s, const StepArgs &a, const SesmPtrs &q, int block,
                        cudaStream_t stream);
// The barotropic viscosity alone at the state (s.U, s.eta[parity]): R_hV of every
// element into out[new element].
cudaError_t launch_viscosity(const DevMesh &m, const DevState &s, const ViscArgs &v, int parity, float2 *out,
                             cudaStream_t stream);
cudaError_t launch_scatter_state(const DevMesh &m, const DevState &s, const double *eta,
                                 const double *U, int parity, cudaStream_t stream);
cudaError_t launch_scatter_forcing(const DevMesh &m, const DevState &s, const double *R,
                                   cudaStream_t stream);
cudaError_t launch_gather_scaled(const DevMesh &m, const float *x, double scale, double *out, cudaStream_t stream);
cudaError_t launch_gather_state(const DevMesh &m, const DevState &s, int parity, double *eta,
                                double *U, double *Umean, cudaStream_t stream);
cudaError_t launch_diagnostics(const DevMesh &m, const DevState &s, const StepArgs &a, int parity,
                               int nblocks, cudaStream_t stream);
int diagnostics_blocks(const DevMesh &m);
// Per-basin volume and energy into out[2 * nbasin] (device).
cudaError_t launch_diagnostics_basins(const DevMesh &m, const DevState &s, const StepArgs &a, int parity,
                                      double *out, cudaStream_t stream);

// Persistent kernel: one launch per baroclinic step (see sesw_kernels.cu).
struct PersistentPlan {
    int slots_per_thread = 0;   // 0: not possible for this mesh
    int threads = 0;
    int cached = 0;             // 1: the patch's static data lives in shared memory
    int stream = 0;             // state and static data in global memory (the streaming kernels):
                                // 1 with the corner indices in shared memory, 2 without
    int blocks_per_sm = 1;
    size_t smem = 0;
};
// Largest patch of a pack: what its shared-memory layout and its plan depend on.
struct PatchMax {
    int slots = 0, local = 0, vertices = 0, halo = 0, csr = 0;
    int deg = 0;   // most incidences (triangle corners) of one vertex
};
// One cooperative launch of a step: blocks [base, base + nblocks) of pack_patch, with the
// plans of both schemes for its largest patch (the SESM plan may be empty).
struct PackPlan {
    int base = 0, nblocks = 0;
    PatchMax mx;
    PersistentPlan plan, plan_sesm;
};
// Consecutive packs [first, last) that one cooperative launch of the SE kernels runs one after
// another: they share the kernel, with the plan and shared-memory layout of their common
// largest patch (mx) and as many blocks as the largest of them.
struct PackGroup {
    int first = 0, last = 0, nblocks = 0;
    PatchMax mx;
    PersistentPlan plan;
};
PersistentPlan persistent_plan(const PatchMax &mx, int blocks_per_sm);
cudaError_t persistent_prepare(const PersistentPlan &plan);
size_t persistent_flag_bytes(int npatch);
cudaError_t launch_persistent(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity,
                              const std::vector<PackGroup> &groups, cudaStream_t stream);
// The SESM scheme for patches too large for its on-chip state (k_persistent_sesm_stream):
// two more slot arrays (DevState::U_x) hold U^{m-2} and U_AB^{m-1}.
// idx_mode: -1 keeps the slots' corner indices in shared memory when they fit, 0 never.
PersistentPlan persistent_plan_sesm_stream(const PatchMax &mx, int blocks_per_sm, int idx_mode = -1);
cudaError_t persistent_prepare_sesm_stream(const PersistentPlan &plan);
cudaError_t launch_persistent_sesm_stream_pack(const DevMesh &m, const DevState &s, const StepArgs &a, int M,
                                               int parity, const PackPlan &pk, int pack_index, cudaStream_t stream);
// Patches too large for the on-chip state (k_persistent_stream): transport, sums and
// static data stay in global memory; only the elevation and the fluxes are on chip.
PersistentPlan persistent_plan_stream(const PatchMax &mx, int blocks_per_sm, int idx_mode = -1);
cudaError_t persistent_prepare_stream(const PersistentPlan &plan);
cudaError_t launch_persistent_stream_group(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity,
                                           const PackGroup &g, cudaStream_t stream);
// The SESM scheme in the persistent form (k_persistent_sesm): cached patches of at most
// 4 x 384 slots and 2 x 384 own vertices; an empty plan when the patches do not fit.
PersistentPlan persistent_plan_sesm(const PatchMax &mx, int blocks_per_sm);
cudaError_t persistent_prepare_sesm(const PersistentPlan &plan);
// Fill m.slot_k from the slots' static data, g and each patch's substep length.
cudaError_t launch_slot_coef(const DevMesh &m, float g, cudaStream_t stream);
cudaError_t launch_persistent_sesm(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity,
                                   const std::vector<PackPlan> &packs, cudaStream_t stream);

struct Surrogate;
void surrogate_release(sesw_ctx *c);

// Message layers on the tensor cores (sesw_tc.cu): K inputs holding bfloat16 values (K = 128
// or 192), 64 outputs. W (K x 64 row-major bf16) is first packed by pack_linear_tc into
// linear_tc_packed_elems(K) elements (the shared-memory image of W^T), which
// launch_msg_layer_tc then reads.
bool linear_tc_supported(int K, int P);
size_t linear_tc_packed_elems(int K);
cudaError_t pack_linear_tc(int K, const __nv_bfloat16 *W, __nv_bfloat16 *packed, cudaStream_t st);
// The inputs of a message layer, formed inside the tensor-core layer from the hidden states:
// kind 0, element rows, Z_e = [h_e, L sum_k dphi_k/dx h_vk, L sum_k dphi_k/dy h_vk] (K = 192);
// kind 1, vertex rows, Z_v = [h_v, sum A_e h_e / sum A_e over the vertex's triangles] (K = 128).
// The layer writes Y = tanh(Z W + b) (unless Y is null) and h_next = h + Y ([N][64] each; h_next
// must not alias the inputs).
struct MsgLayerArgs {
    int kind;                   // 0 element rows, 1 vertex rows
    int N;                      // rows
    const int4 *etri;           // element corners
    const float4 *egrad;        // element basis gradients (dphi0/dx, dphi0/dy, dphi1/dx, dphi1/dy)
    float L;                    // length scale of the element message
    const int *voff, *vinc;     // vertex incidences (element << 2 | corner), CSR
    const float *earea, *vinvA; // element areas; 1 / sum of each vertex's element areas
    const float *hself;         // hidden state of the rows' own kind
    const float *hother;        // hidden state of the other kind
    float *Y, *hnext;
};
cudaError_t launch_msg_layer_tc(const MsgLayerArgs &a, const __nv_bfloat16 *packed, const float *bias,
                                unsigned *status, cudaStream_t st);
// Backward of such a layer on the tensor cores, dA (FP32) split into two bfloat16 parts:
// partial sums of the weight gradient sum_n Z[n][i] dA[n][j] and of the bias gradient over
// rows_per_cta rows each (a multiple of 64; layout of k_reduce_partials), and the input
// gradient dZ[n][i] = sum_j dA[n][j] W[i][j] (W: K x 64 bfloat16, row-major). K = 128 or 192.
cudaError_t launch_wgrad_tc(int N, int K, int rows_per_cta, const float *Z, const float *dA, float *partial,
                            unsigned *status, cudaStream_t st);
cudaError_t launch_dgrad_tc(int N, int K, const float *dA, const __nv_bfloat16 *W, float *dZ, unsigned *status,
                            cudaStream_t st);

}  // namespace sesw

// The context behind the C-ABI handle.
struct sesw_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    sesw_alloc_fn alloc = nullptr;
    sesw_free_fn free_fn = nullptr;
    void *user = nullptr;
    std::string err;
    int patch_vertices = 256;
    int block_threads = 256;
    int mode_req = SESW_MODE_AUTO, mode = SESW_MODE_GRAPH;
    int blocks_per_sm = 0;         // persistent mode; 0 = try 2, then 1
    int form = SESW_FORM_AUTO;     // persistent mode: which kernel a pack runs (sesw_set_persistent_form)
    int large_bps = 0;             // batches: resident blocks per SM of the large basins' packs (0: blocks_per_sm)
    int large_form = -1;           // batches: kernel form of the large basins' packs (-1: form)
    sesw::PersistentPlan plan;
    sesw::PersistentPlan plan_sesm;   // the SESM scheme's plan (empty: graph mode only)
    std::vector<sesw::PackPlan> packs;   // persistent mode: the packs of a step (one launch each for SESM)
    std::vector<sesw::PackGroup> groups; // persistent mode: the launches of an SE step
    bool persist_graph_ok = true;
    bool have_mesh = false, have_params = false;
    sesw::DevMesh dm;
    sesw::DevState ds;
    std::vector<std::pair<void *, size_t>> allocs;
    int64_t device_bytes = 0;
    sesw_params params{};
    sesw::StepArgs args{};
    int parity = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int diag_blocks = 1;
    double grad_gram_max_h = 0.0;
    double courant_max = 0.0, courant_limit = 0.0;
    int npatch = 0, nslot = 0, max_patch_slots = 0, patch_vertices_used = 0;
    int nbasin = 1;
    std::vector<int> patch_basin;
    std::vector<double> basin_stiffness;
    std::vector<double> basin_visc_stiffness;
    std::vector<float> patch_dt_host;
    double visc_number = 0.0;      // largest dt A_bg visc_stiffness over the basins
    bool visc_on = false;          // barotropic viscosity in the step (graph mode, SE)
    sesw::ViscArgs vargs{};
    float2 *visc_out = nullptr;    // [ne] scratch of sesw_viscosity (allocated on first use)
    float *W_buf = nullptr;        // [nv] freshwater flux (allocated on first use)
    float *eta_sum_buf = nullptr;  // [nv] sum of the substep elevations (allocated on first use)
    // asynchronous host transfers: copy streams and double-buffered device staging
    cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
    cudaEvent_t in_done[2] = {}, in_free[2] = {}, out_ready[2] = {}, out_done[2] = {};
    double *stage_in[2] = {nullptr, nullptr};    // [2 ne] forcing in transit
    double *stage_out[2] = {nullptr, nullptr};   // [nv + 4 ne] state in transit
    unsigned *status_h = nullptr;                // [2] pinned: the status word as of each buffer's last download
    int in_idx = 0, out_idx = 0;
    uint64_t out_seq = 0;
    bool have_W = false;
    sesw::Surrogate *sur = nullptr;
};

namespace sesw {
// Helpers of sesw_api.cpp for other translation units.
int ctx_fail(sesw_ctx *c, int code, const std::string &msg);
int ctx_fail_cuda(sesw_ctx *c, const char *what, cudaError_t e);
void *ctx_alloc(sesw_ctx *c, size_t bytes);
int ctx_enqueue_step(sesw_ctx *c);
}  // namespace sesw
