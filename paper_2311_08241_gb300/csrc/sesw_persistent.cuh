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
// Incidences of a vertex in the padded form (PArgs::inc8): at most this many per vertex.
constexpr int kIncWidth = 8;

struct PArgs {
    const int *patch_slot, *patch_own, *patch_int, *patch_v, *patch_halo, *halo_v;
    const int *vcsr_off;
    const uint32_t *vcsr;
    const int4 *sv;
    const ushort4 *sl;
    const float4 *sg, *sc;
    const float4 *sk;          // step coefficients of each slot (DevMesh::slot_k)
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
    int pack_base, pack_index;   // launches of one pack (the SESM kernels)
    const int *pack_off;         // [npack + 1] ranges of pack_patch
    int pack_first, pack_last;   // launches of a group of packs (the SE kernels)
    StepArgs a;
    int M, npatch;
    // shared-memory carve-up (CACHED), in bytes from the dynamic shared base
    int off_flux, off_g, off_c, off_r, off_l, off_off, off_csr, off_inv, off_halo;
    // inc8: the cached incidences are one row of 8 16-bit byte offsets per own vertex (into the
    // dynamic shared memory: the corner fluxes, padded with a zero word) at off_off, in place of
    // the CSR (offsets at off_off, entries at off_csr); zero_off: the zero word's byte offset
    int inc8, zero_off;
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


// Copy the incidences of a patch's own vertices into shared memory (cached layouts): with
// P.inc8, one row of kIncWidth 16-bit byte offsets (inc8 = 1) or word indices (inc8 = 2) per
// vertex, pointing at its corner fluxes in incidence order and padded with the zero word; else
// the CSR with flux indices 3 * slot + corner. Also clears the zero word. The caller synchronises the block afterwards.
__device__ __forceinline__ void cache_incidences(const PArgs &P, unsigned char *smem_raw, int v0, int nown)
{
    const int c0 = P.vcsr_off[v0], ncsr = P.vcsr_off[v0 + nown] - c0;
    if (P.inc8) {
        uint4 *rows = reinterpret_cast<uint4 *>(smem_raw + P.off_off);
        for (int i = threadIdx.x; i < nown; i += blockDim.x) {
            const int k0 = P.vcsr_off[v0 + i], deg = P.vcsr_off[v0 + i + 1] - k0;
            unsigned h[kIncWidth];
#pragma unroll
            for (int k = 0; k < kIncWidth; k++) {
                unsigned off = (unsigned)P.zero_off;
                if (k < deg) {
                    const uint32_t q = P.vcsr[k0 + k];
                    off = (unsigned)P.off_flux + 4u * (3u * (q >> 2) + (q & 3u));
                }
                h[k] = P.inc8 == 2 ? off >> 2 : off;
            }
            rows[i] = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
        }
        if (threadIdx.x == 0) *reinterpret_cast<float *>(smem_raw + P.zero_off) = 0.0f;
    } else {
        unsigned short *s_off = reinterpret_cast<unsigned short *>(smem_raw + P.off_off);
        unsigned short *s_csr = reinterpret_cast<unsigned short *>(smem_raw + P.off_csr);
        for (int i = threadIdx.x; i <= nown; i += blockDim.x) s_off[i] = (unsigned short)(P.vcsr_off[v0 + i] - c0);
        for (int k = threadIdx.x; k < ncsr; k += blockDim.x) {
            const uint32_t q = P.vcsr[c0 + k];
            s_csr[k] = (unsigned short)(3u * (q >> 2) + (q & 3u));
        }
    }
}

// Sum of the corner fluxes of own vertex i in its incidence order (cached layouts; see
// cache_incidences). The padded form adds zeros after the last incidence, which leaves the
// sum unchanged.
__device__ __forceinline__ float cached_flux_sum(const PArgs &P, const unsigned char *smem_raw, int i)
{
    float sum = 0.0f;
    if (P.inc8 == 1) {
        const uint4 q = reinterpret_cast<const uint4 *>(smem_raw + P.off_off)[i];
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            sum = __fadd_rn(sum, *reinterpret_cast<const float *>(smem_raw + (w[k] & 0xffffu)));
            sum = __fadd_rn(sum, *reinterpret_cast<const float *>(smem_raw + (w[k] >> 16)));
        }
    } else if (P.inc8 == 2) {
        const uint4 q = reinterpret_cast<const uint4 *>(smem_raw + P.off_off)[i];
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
        const float *words = reinterpret_cast<const float *>(smem_raw);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            sum = __fadd_rn(sum, words[w[k] & 0xffffu]);
            sum = __fadd_rn(sum, words[w[k] >> 16]);
        }
    } else {
        const unsigned short *s_off = reinterpret_cast<const unsigned short *>(smem_raw + P.off_off);
        const unsigned short *s_csr = reinterpret_cast<const unsigned short *>(smem_raw + P.off_csr);
        const float *sflux = reinterpret_cast<const float *>(smem_raw + P.off_flux);
        const int k1 = s_off[i + 1];
        for (int k = s_off[i]; k < k1; k++) sum = __fadd_rn(sum, sflux[s_csr[k]]);
    }
    return sum;
}

inline size_t flag_bytes(int npatch) { return sizeof(unsigned) * (2 * (size_t)npatch + 1) * kFlagStride; }


struct SmemLayout {
    int off_flux, off_g, off_c, off_r, off_l, off_off, off_csr, off_inv, off_halo;
    int inc8, zero_off;
    size_t total_plain;     // elevation, corner fluxes and the zero word
    size_t total_vcached;   // ... and the vertices' data: 1/A_v, halo ids, incidences
    size_t total_cached;    // ... and the slots' static data
};

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory layout of a patch: [elevation of own and halo vertices | corner fluxes, zero
// word | 1/A_v, halo ids, incidences | per slot: gradients, coefficients, forcing, corners].
// The kernels that keep everything on chip use the whole layout (CACHED = 1), those for larger
// patches the part up to the incidences (CACHED = 2: the slots' static data then come from L2),
// the streaming kernels only the first part.
inline SmemLayout smem_layout(const PatchMax &m)
{
    SmemLayout L;
    size_t o = align16(sizeof(float) * (size_t)m.local);
    L.off_flux = (int)o;
    // the corner fluxes, then one zero word (the padding target of the padded incidence rows)
    L.zero_off = (int)(o + sizeof(float) * 3 * (size_t)m.slots);
    o = align16(o + sizeof(float) * (3 * (size_t)m.slots + 1));
    L.total_plain = o;
    L.off_inv = (int)o;
    o = align16(o + sizeof(float) * (size_t)m.vertices);
    L.off_halo = (int)o;
    o = align16(o + sizeof(int) * (size_t)m.halo);
    L.off_off = (int)o;
    const size_t csr_end = align16(align16(o + sizeof(unsigned short) * ((size_t)m.vertices + 1)) +
                                   sizeof(unsigned short) * (size_t)m.csr);
    L.off_csr = (int)align16(o + sizeof(unsigned short) * ((size_t)m.vertices + 1));
    // padded rows when every vertex has at most kIncWidth incidences: 16-bit byte offsets of the
    // corner fluxes when they fit 16 bits (inc8 = 1), else 16-bit word indices (inc8 = 2); they
    // take the place of the CSR
    L.inc8 = m.deg > kIncWidth ? 0 : (L.zero_off + 4 <= 65535 ? 1 : (L.zero_off / 4 + 1 <= 65535 ? 2 : 0));
    const size_t inc_end = o + sizeof(unsigned short) * kIncWidth * (size_t)m.vertices;
    o = L.inc8 ? align16(inc_end) : csr_end;
    L.total_vcached = o;
    L.off_g = (int)o;
    o += sizeof(float4) * (size_t)m.slots;
    L.off_c = (int)o;
    o += sizeof(float4) * (size_t)m.slots;
    L.off_r = (int)o;
    o = align16(o + sizeof(float2) * (size_t)m.slots);
    L.off_l = (int)o;
    o = align16(o + sizeof(ushort4) * (size_t)m.slots);
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
    P.sk = m.slot_k;
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
    P.inc8 = L.inc8;
    P.zero_off = L.zero_off;
    P.pack_patch = m.pack_patch;
    P.pack_base = 0;
    P.pack_index = 0;
    P.pack_off = m.pack_off_d;
    P.pack_first = 0;
    P.pack_last = 0;
    return P;
}

}  // namespace

}  // namespace sesw
