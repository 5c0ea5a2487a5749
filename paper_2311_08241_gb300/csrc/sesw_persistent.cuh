// Shared parts of the persistent step kernels of libsesw (sm_103a): kernel arguments,
// the tagged exchange of halo values through L2 and the shared-memory layout of a patch.
// Included by sesw_persistent.cu (the SE substep of Eq. 4.10), sesw_persistent_stream.cu
// (the same for patches whose state is streamed from L2) and sesw_persistent_sesm.cu (the
// SESM substep of Eqs. 4.7-4.8).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "sesw_device.cuh"
#include "sesw_internal.h"

namespace sesw {

namespace {

// The persistent kernels run one cooperative launch per baroclinic step, one block per
// patch, all blocks resident.
//
// Exchange protocol. Every exchanged value (the elevation, or for SESM its AM4
// combination) is one 64-bit word holding a tag (high
// half) and its value (low half), written and read as a single relaxed access at GPU
// scope. The tag of substep m is base + m, where base is this launch's tag base. A
// reader uses a word only when its tag is the one it needs, re-reading it (bounded)
// otherwise, so it can never take a stale or a torn value, and no flag, fence or
// block-wide barrier is needed for the exchange. Within a launch, a block overwrites a
// parity buffer (tag m with m + 2) only after its substep m + 1, which needed every
// neighbour's tag-(m + 1) values; a neighbour writes those only after its own substep
// m, in which it read the tag-m values (the neighbour relation is symmetric: each patch
// reads halo values from every patch that reads from it). Between launches, the last
// block to leave advances the base by M + 1 (one word per pack in the flag buffer), so
// every word left by an earlier launch carries a tag that this launch never waits for
// and the buffers need no clearing. Tags wrap modulo 2^32; a wrapped tag could only
// match a word that no launch has rewritten since, and every launch rewrites every word
// that is read.
struct PArgs {
    const int *patch_slot, *patch_own, *patch_int, *patch_v, *patch_halo, *halo_v;
    const int *vcsr_off;
    const uint32_t *vcsr;
    const int4 *sv;
    const ushort4 *sl;
    const float4 *sg, *sc;
    const float2 *R;
    float2 *U, *Umean;
    const float *inv_av;
    const float *patch_dt;
    const float *eta_in;
    float *eta_out;
    float *eta_sum;         // null, or sum over the substeps of eta^0 .. eta^{M-1} (own vertices)
    const float *W;         // null, or the freshwater flux of each vertex (Eq. 4.5)
    unsigned long long *xb[2];  // tagged elevation words (tag << 32 | float bits), per substep parity
    unsigned *flags;        // line 0: abort word; line 1 + 2k: tag base of pack k; line 2 + 2k: its exit count
    unsigned *status;
    const int *pack_patch;  // patch of each block: pack_patch[pack_base + blockIdx.x]
    int pack_base, pack_index;
    StepArgs a;
    int M, npatch;
    // shared-memory carve-up (CACHED), in bytes from the dynamic shared base
    int off_flux, off_g, off_c, off_r, off_l, off_off, off_csr, off_inv, off_halo;
};

__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_relaxed_gpu_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The flag buffer holds 2 npatch + 1 lines of 128 bytes (at most one pack per patch).
constexpr int kFlagStride = 32;

// The halo elevation of vertex v with tag `tag`, given the exchange word `w` already
// read from xs[v]: re-read until the word carries that tag. A wait that exceeds the
// budget (or finds the abort word set to this launch's `abort_val`) gives up: it sets
// the timeout bit and the abort word, which makes every other wait of the launch give
// up too, and clears `ok`; the value returned then is meaningless. (The first reads of
// a slot's corners are issued together by the caller, so that their latencies overlap.)
__device__ __forceinline__ float halo_eta(const PArgs &P, const unsigned long long *xs, int v,
                                          unsigned long long w, unsigned tag, unsigned abort_val, bool &ok)
{
    if ((unsigned)(w >> 32) == tag) return __uint_as_float((unsigned)w);
    const unsigned *abort_word = P.flags;
    const long long t0 = clock64();
    while (ok) {
        __nanosleep(20);
        w = ld_relaxed_gpu_u64(xs + v);
        if ((unsigned)(w >> 32) == tag) return __uint_as_float((unsigned)w);
        if (ld_relaxed_gpu(abort_word) == abort_val || clock64() - t0 > P.a.wait_cycles) {
            ok = false;
            atomicOr(P.status, 2u);
            atomicExch(const_cast<unsigned *>(abort_word), abort_val);
        }
    }
    return 0.0f;
}


inline size_t flag_bytes(int npatch) { return sizeof(unsigned) * (2 * (size_t)npatch + 1) * kFlagStride; }


struct SmemLayout {
    int off_flux, off_g, off_c, off_r, off_l, off_off, off_csr, off_inv, off_halo;
    size_t total_plain, total_cached;
};

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

inline SmemLayout smem_layout(const PatchMax &m)
{
    SmemLayout L;
    size_t o = align16(sizeof(float) * (size_t)m.local);
    L.off_flux = (int)o;
    o = align16(o + sizeof(float) * 3 * (size_t)m.slots);
    L.total_plain = o;
    L.off_g = (int)o;
    o += sizeof(float4) * (size_t)m.slots;
    L.off_c = (int)o;
    o += sizeof(float4) * (size_t)m.slots;
    L.off_r = (int)o;
    o = align16(o + sizeof(float2) * (size_t)m.slots);
    L.off_l = (int)o;
    o = align16(o + sizeof(ushort4) * (size_t)m.slots);
    L.off_inv = (int)o;
    o = align16(o + sizeof(float) * (size_t)m.vertices);
    L.off_halo = (int)o;
    o = align16(o + sizeof(int) * (size_t)m.halo);
    L.off_off = (int)o;
    o = align16(o + sizeof(unsigned short) * ((size_t)m.vertices + 1));
    L.off_csr = (int)o;
    o = align16(o + sizeof(unsigned short) * (size_t)m.csr);
    L.total_cached = o;
    return L;
}


inline PArgs make_pargs(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity, const PatchMax &mx)
{
    PArgs P;
    P.patch_slot = m.patch_slot;
    P.patch_own = m.patch_own;
    P.patch_int = m.patch_int;
    P.patch_v = m.patch_v;
    P.patch_halo = m.patch_halo;
    P.halo_v = m.halo_v;
    P.vcsr_off = m.vcsr_off;
    P.vcsr = m.vcsr;
    P.sv = m.slot_v;
    P.sl = m.slot_l;
    P.sg = m.slot_g;
    P.sc = m.slot_c;
    P.R = s.R;
    P.U = s.U;
    P.Umean = s.Umean;
    P.inv_av = m.inv_av;
    P.patch_dt = m.patch_dt;
    P.eta_in = s.eta[parity];
    P.eta_out = s.eta[parity ^ 1];
    P.eta_sum = s.eta_sum;
    P.W = s.W;
    P.xb[0] = reinterpret_cast<unsigned long long *>(s.xbuf[0]);
    P.xb[1] = reinterpret_cast<unsigned long long *>(s.xbuf[1]);
    P.flags = s.flags;
    P.status = s.status;
    P.a = a;
    P.M = M;
    P.npatch = m.npatch;
    const SmemLayout L = smem_layout(mx);
    P.off_flux = L.off_flux;
    P.off_g = L.off_g;
    P.off_c = L.off_c;
    P.off_r = L.off_r;
    P.off_l = L.off_l;
    P.off_off = L.off_off;
    P.off_csr = L.off_csr;
    P.off_inv = L.off_inv;
    P.off_halo = L.off_halo;
    P.pack_patch = m.pack_patch;
    P.pack_base = 0;
    P.pack_index = 0;
    return P;
}

}  // namespace

}  // namespace sesw
