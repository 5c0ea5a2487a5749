// Internal declarations shared by the host side (mesh prep, C-ABI) and the CUDA
// kernels of libsesw. Not part of the public interface (include/sesw.h).
#pragma once

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
    std::vector<int4> slot_v;      // corners (new vertex ids); .w = element id, or -1-element for guests
    std::vector<float4> slot_g;    // (dphi0/dx, dphi0/dy, dphi1/dx, dphi1/dy); dphi2 = -dphi0 - dphi1
    std::vector<float4> slot_c;    // (A_e, H0_e, f_e, 0)
    std::vector<int> vcsr_off;     // [nv+1] incidence list of each vertex
    std::vector<uint32_t> vcsr;    // (local slot << 2) | corner, local to the vertex's patch
    std::vector<float> inv_av;     // 1 / median-dual area
    std::vector<double> area_v;    // median-dual area (FP64, for diagnostics)
    std::vector<double> area_e;    // element area (FP64), new element order
    std::vector<double> h0_e;      // element rest depth (FP64), new element order
    double grad_gram_max_h = 0.0;  // upper bound of lambda_max(-div H0 grad) (m/s^2 units without g)
};

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
    int *vcsr_off = nullptr;
    uint32_t *vcsr = nullptr;
    float *inv_av = nullptr;
    double *area_v = nullptr;
    int *vperm = nullptr;
    int *eperm = nullptr;
    int *elem_slot = nullptr;      // new element -> owner slot
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
};

struct StepArgs {
    float g, theta, dt, half_dt, inv_M, eta_bound;
    int nonlinear_h;
    double g64;
};

// Kernel launchers (sesw_kernels.cu). All enqueue on `stream` and return the
// launch error.
cudaError_t launch_substep(const DevMesh &m, const DevState &s, const StepArgs &a, int parity,
                           int block, cudaStream_t stream);
cudaError_t substep_smem_attr(const DevMesh &m);
cudaError_t launch_step_epilogue(const DevMesh &m, const DevState &s, const StepArgs &a,
                                 cudaStream_t stream);
cudaError_t launch_scatter_state(const DevMesh &m, const DevState &s, const double *eta,
                                 const double *U, int parity, cudaStream_t stream);
cudaError_t launch_scatter_forcing(const DevMesh &m, const DevState &s, const double *R,
                                   cudaStream_t stream);
cudaError_t launch_gather_state(const DevMesh &m, const DevState &s, int parity, double *eta,
                                double *U, double *Umean, cudaStream_t stream);
cudaError_t launch_diagnostics(const DevMesh &m, const DevState &s, const StepArgs &a, int parity,
                               int nblocks, cudaStream_t stream);
int diagnostics_blocks(const DevMesh &m);

}  // namespace sesw
