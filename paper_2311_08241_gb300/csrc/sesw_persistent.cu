// The persistent step kernel of libsesw (sm_103a): one cooperative launch runs all M
// substeps of Eq. (4.10) of a baroclinic step, with the time-mean transport of Eq.
// (4.12) and the freshwater flux of Eq. (4.5).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sesw_device.cuh"
#include "sesw_internal.h"

namespace sesw {

namespace {

// ---------------------------------------------------------------------------------
// Persistent kernel: one launch per baroclinic step, one block per patch, all blocks
// resident (cooperative launch). A block keeps the elevation of its own and halo
// vertices and the per-corner fluxes in shared memory, and the transport and the
// compensated flux sum of its slots in registers, for all M substeps. When it fits
// (CACHED), the patch's static slot data, incidence lists, 1/A_v and halo index list
// are also copied to shared memory once per step.
//
// Substep m: update the interior slots (corners all own vertices); update the other
// slots, reading the halo elevation from the exchange buffer of parity m; vertex pass;
// write the own vertices' new elevation to the exchange buffer of parity m+1.
//
// Exchange protocol. Every exchanged elevation is one 64-bit word holding a tag (high
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
//
// Vertex order. Mesh preparation puts the vertices that other patches read first in
// each patch, so the vertex pass publishes them in its first round; the halo words of a
// thread's last-round slot are then requested right after its first element round and
// have usually arrived by the time the slot is updated.
struct PArgs {
    const int *patch_slot, *patch_own, *patch_int, *patch_v, *patch_halo, *halo_v, *patch_nbr, *nbr;
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

// Element update of one slot (Eq. 4.10, first row, and the theta-weighted flux);
// coef = (dt A_e, g H0_e, f dt / 2, 1 / (1 + (f dt / 2)^2)).
template <int NONLIN>
__device__ __forceinline__ void element_update(const float e0, const float e1, const float e2, const float4 g,
                                               const float4 coef, const float2 r, float2 &u, float2 &shi,
                                               float2 &slo, bool owned, float *flux3, float theta,
                                               float one_p_theta, float dt, float gconst)
{
    const float d0 = e0 - e2, d1 = e1 - e2;
    const float gx = d0 * g.x + d1 * g.z;
    const float gy = d0 * g.y + d1 * g.w;
    float gH = coef.y;
    if (NONLIN) gH += gconst * ((e0 + e1 + e2) * (1.0f / 3.0f));
    const float aa = coef.z;
    const float rx = u.x + aa * u.y + dt * (r.x - gH * gx);
    const float ry = u.y - aa * u.x + dt * (r.y - gH * gy);
    const float nx = (rx + aa * ry) * coef.w;
    const float ny = (ry - aa * rx) * coef.w;
    const float fx = one_p_theta * nx - theta * u.x;
    const float fy = one_p_theta * ny - theta * u.y;
    u = make_float2(nx, ny);
    if (owned) {
        two_sum_acc(shi.x, slo.x, fx);
        two_sum_acc(shi.y, slo.y, fy);
    }
    const float c0 = coef.x * (fx * g.x + fy * g.y);
    const float c1 = coef.x * (fx * g.z + fy * g.w);
    flux3[0] = c0;
    flux3[1] = c1;
    flux3[2] = -(c0 + c1);
}

__device__ __forceinline__ float4 slot_coef(const float4 c, const StepArgs &a, float dt)
{
    const float aa = c.z * (0.5f * dt);
    return make_float4(dt * c.x, a.g * c.y, aa, 1.0f / (1.0f + aa * aa));
}

// EXTRA: the optional per-vertex terms (freshwater flux, step-mean elevation) may be set;
// the instantiation without them carries neither load nor branch.
template <int SPT, int NONLIN, int CACHED, int EXTRA>
__global__ void __launch_bounds__(1024, 1) k_persistent(PArgs P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_abort;
    const int p = P.pack_patch[P.pack_base + blockIdx.x];
    const int T = blockDim.x;
    const int s0 = P.patch_slot[p], ns = P.patch_slot[p + 1] - s0;
    const int nown_s = P.patch_own[p], nint = P.patch_int[p];
    const int v0 = P.patch_v[p], nown = P.patch_v[p + 1] - v0;
    const int hb = P.patch_halo[p], nhalo = P.patch_halo[p + 1] - hb;
    const int c0 = P.vcsr_off[v0], ncsr = P.vcsr_off[v0 + nown] - c0;
    const StepArgs a = P.a;
    const float dt = P.patch_dt[p];
    unsigned *base_word = P.flags + (size_t)(1 + 2 * P.pack_index) * kFlagStride;
    unsigned *exit_count = base_word + kFlagStride;
    const unsigned base = ld_relaxed_gpu(base_word);
    const unsigned abort_val = base + 1u == 0u ? 1u : base + 1u;   // never 0, unique per launch

    float *seta = reinterpret_cast<float *>(smem_raw);
    float *sflux = reinterpret_cast<float *>(smem_raw + P.off_flux);
    float4 *s_g = reinterpret_cast<float4 *>(smem_raw + P.off_g);
    float4 *s_c = reinterpret_cast<float4 *>(smem_raw + P.off_c);
    float2 *s_r = reinterpret_cast<float2 *>(smem_raw + P.off_r);
    ushort4 *s_l = reinterpret_cast<ushort4 *>(smem_raw + P.off_l);
    unsigned short *s_off = reinterpret_cast<unsigned short *>(smem_raw + P.off_off);
    unsigned short *s_csr = reinterpret_cast<unsigned short *>(smem_raw + P.off_csr);
    float *s_inv = reinterpret_cast<float *>(smem_raw + P.off_inv);
    int *s_halo = reinterpret_cast<int *>(smem_raw + P.off_halo);

    for (int i = threadIdx.x; i < nown; i += T) seta[i] = P.eta_in[v0 + i];
    for (int i = threadIdx.x; i < nhalo; i += T) seta[nown + i] = P.eta_in[P.halo_v[hb + i]];
    if (CACHED) {
        for (int i = threadIdx.x; i < ns; i += T) {
            s_g[i] = P.sg[s0 + i];
            s_c[i] = slot_coef(P.sc[s0 + i], a, dt);
            s_r[i] = P.R[s0 + i];
            s_l[i] = P.sl[s0 + i];
        }
        for (int i = threadIdx.x; i <= nown; i += T) s_off[i] = (unsigned short)(P.vcsr_off[v0 + i] - c0);
        // cached incidence entries hold the flux index 3 * slot + corner directly
        for (int k = threadIdx.x; k < ncsr; k += T) {
            const uint32_t q = P.vcsr[c0 + k];
            s_csr[k] = (unsigned short)(3u * (q >> 2) + (q & 3u));
        }
        for (int i = threadIdx.x; i < nown; i += T) s_inv[i] = P.inv_av[v0 + i];
        for (int i = threadIdx.x; i < nhalo; i += T) s_halo[i] = P.halo_v[hb + i];
    }
    if (threadIdx.x == 0) s_abort = 0;
    float2 u[SPT], shi[SPT], slo[SPT];
#pragma unroll
    for (int j = 0; j < SPT; j++) {
        const int i = threadIdx.x + j * T;
        u[j] = i < ns ? P.U[s0 + i] : make_float2(0.0f, 0.0f);
        shi[j] = make_float2(0.0f, 0.0f);
        slo[j] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();

    const float one_p_theta = 1.0f + a.theta;
    // Element update of the slots with local index in [lo, hi). Corner elevations of
    // own vertices come from shared memory; with `halo_src` set, those of halo vertices
    // are read from that exchange buffer with tag `tag`. Used for the first substep (all
    // halo values are in shared memory then) and, with one slot per thread, for all.
    bool ok = true;
    auto elements = [&](int lo, int hi, const unsigned long long *halo_src, unsigned tag) {
#pragma unroll
        for (int j = 0; j < SPT; j++) {
            const int i = threadIdx.x + j * T;
            if (i >= lo && i < hi) {
                float4 g, coef;
                float2 r;
                ushort4 l;
                if (CACHED) {
                    g = s_g[i];
                    coef = s_c[i];
                    r = s_r[i];
                    l = s_l[i];
                } else {
                    g = P.sg[s0 + i];
                    coef = slot_coef(P.sc[s0 + i], a, dt);
                    r = P.R[s0 + i];
                    l = P.sl[s0 + i];
                }
                float e0, e1, e2;
                if (halo_src) {
                    const int *hid = CACHED ? s_halo : P.halo_v + hb;
                    const int h0 = l.x < nown ? -1 : hid[l.x - nown], h1 = l.y < nown ? -1 : hid[l.y - nown],
                              h2 = l.z < nown ? -1 : hid[l.z - nown];
                    const unsigned long long w0 = h0 < 0 ? 0ull : ld_relaxed_gpu_u64(halo_src + h0);
                    const unsigned long long w1 = h1 < 0 ? 0ull : ld_relaxed_gpu_u64(halo_src + h1);
                    const unsigned long long w2 = h2 < 0 ? 0ull : ld_relaxed_gpu_u64(halo_src + h2);
                    e0 = h0 < 0 ? seta[l.x] : halo_eta(P, halo_src, h0, w0, tag, abort_val, ok);
                    e1 = h1 < 0 ? seta[l.y] : halo_eta(P, halo_src, h1, w1, tag, abort_val, ok);
                    e2 = h2 < 0 ? seta[l.z] : halo_eta(P, halo_src, h2, w2, tag, abort_val, ok);
                } else {
                    e0 = seta[l.x];
                    e1 = seta[l.y];
                    e2 = seta[l.z];
                }
                element_update<NONLIN>(e0, e1, e2, g, coef, r, u[j], shi[j], slo[j], i < nown_s, sflux + 3 * i,
                                       a.theta, one_p_theta, dt, a.g);
            }
        }
    };

    // element update of slot i (round j of this thread) from its corner elevations; the
    // round's registers are selected by comparison (j is a constant once unrolled)
    auto slot_update = [&](int j, int i, float e0, float e1, float e2) {
        float4 g, coef;
        float2 r;
        if (CACHED) {
            g = s_g[i];
            coef = s_c[i];
            r = s_r[i];
        } else {
            g = P.sg[s0 + i];
            coef = slot_coef(P.sc[s0 + i], a, dt);
            r = P.R[s0 + i];
        }
        float2 uu = u[0], sh = shi[0], sl = slo[0];
#pragma unroll
        for (int q = 1; q < SPT; q++)
            if (q == j) { uu = u[q]; sh = shi[q]; sl = slo[q]; }
        element_update<NONLIN>(e0, e1, e2, g, coef, r, uu, sh, sl, i < nown_s, sflux + 3 * i, a.theta,
                               one_p_theta, dt, a.g);
#pragma unroll
        for (int q = 0; q < SPT; q++)
            if (q == j) { u[q] = uu; shi[q] = sh; slo[q] = sl; }
    };

    // Slots updated first: whole rounds of interior slots (one per thread each), so that
    // no thread does more rounds in total than ceil(ns / T); the interior slots left over
    // go with the boundary slots, whose halo reads may have to wait for a neighbour.
    const int npre = nint >= T ? (nint / T) * T : nint;
    for (int m = 0; m < P.M; m++) {
        if (m == 0 || SPT == 1) {
            if (m == 0) {
                elements(0, ns, nullptr, 0u);
            } else {
                elements(0, npre, nullptr, 0u);
                elements(npre, ns, P.xb[m & 1], base + (unsigned)m);
            }
        } else {
            // The last round's slot, when it is not a whole-round interior one, has its
            // halo words requested right after the first round, so that their L2 round
            // trip overlaps the rounds in between; the other boundary slots issue their
            // three reads together when they come.
            const unsigned long long *xs = P.xb[m & 1];
            const int *hid = CACHED ? s_halo : P.halo_v + hb;
            unsigned long long q0 = 0ull, q1 = 0ull, q2 = 0ull;
            const int ilast = threadIdx.x + (SPT - 1) * T;
            const bool early = ilast >= npre && ilast < ns;
#pragma unroll
            for (int j = 0; j < SPT; j++) {
                const int i = threadIdx.x + j * T;
                if (j == SPT - 1) {
                    if (early) {
                        const ushort4 l = CACHED ? s_l[i] : P.sl[s0 + i];
                        const int h0 = l.x < nown ? -1 : hid[l.x - nown], h1 = l.y < nown ? -1 : hid[l.y - nown],
                                  h2 = l.z < nown ? -1 : hid[l.z - nown];
                        const float e0 = h0 < 0 ? seta[l.x] : halo_eta(P, xs, h0, q0, base + (unsigned)m, abort_val, ok);
                        const float e1 = h1 < 0 ? seta[l.y] : halo_eta(P, xs, h1, q1, base + (unsigned)m, abort_val, ok);
                        const float e2 = h2 < 0 ? seta[l.z] : halo_eta(P, xs, h2, q2, base + (unsigned)m, abort_val, ok);
                        slot_update(j, i, e0, e1, e2);
                    } else if (i < npre) {
                        const ushort4 l = CACHED ? s_l[i] : P.sl[s0 + i];
                        slot_update(j, i, seta[l.x], seta[l.y], seta[l.z]);
                    }
                } else if (i < ns) {
                    const ushort4 l = CACHED ? s_l[i] : P.sl[s0 + i];
                    if (i < npre) {
                        slot_update(j, i, seta[l.x], seta[l.y], seta[l.z]);
                    } else {
                        const int h0 = l.x < nown ? -1 : hid[l.x - nown], h1 = l.y < nown ? -1 : hid[l.y - nown],
                                  h2 = l.z < nown ? -1 : hid[l.z - nown];
                        const unsigned long long w0 = h0 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h0);
                        const unsigned long long w1 = h1 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h1);
                        const unsigned long long w2 = h2 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h2);
                        const float e0 = h0 < 0 ? seta[l.x] : halo_eta(P, xs, h0, w0, base + (unsigned)m, abort_val, ok);
                        const float e1 = h1 < 0 ? seta[l.y] : halo_eta(P, xs, h1, w1, base + (unsigned)m, abort_val, ok);
                        const float e2 = h2 < 0 ? seta[l.z] : halo_eta(P, xs, h2, w2, base + (unsigned)m, abort_val, ok);
                        slot_update(j, i, e0, e1, e2);
                    }
                }
                if (j == 0 && early) {
                    const ushort4 l = CACHED ? s_l[ilast] : P.sl[s0 + ilast];
                    const int h0 = l.x < nown ? -1 : hid[l.x - nown], h1 = l.y < nown ? -1 : hid[l.y - nown],
                              h2 = l.z < nown ? -1 : hid[l.z - nown];
                    if (h0 >= 0) q0 = ld_relaxed_gpu_u64(xs + h0);
                    if (h1 >= 0) q1 = ld_relaxed_gpu_u64(xs + h1);
                    if (h2 >= 0) q2 = ld_relaxed_gpu_u64(xs + h2);
                }
            }
        }
        if (m > 0 && !ok) s_abort = 1;
        __syncthreads();
        if (s_abort) break;

        // vertex pass; the new elevation of own vertices also goes to the exchange buffer
        const bool more = m + 1 < P.M;
        unsigned long long *xout = P.xb[(m + 1) & 1];
        const unsigned long long tag_out = (unsigned long long)(base + (unsigned)(m + 1)) << 32;
        const bool publish = more && p != a.silent_patch;
        bool bad = false;
        for (int i = threadIdx.x; i < nown; i += T) {
            float sum = 0.0f, inv;
            if (CACHED) {
                const int k1 = s_off[i + 1];
                for (int k = s_off[i]; k < k1; k++) sum += sflux[s_csr[k]];
                inv = s_inv[i];
            } else {
                const int k1 = P.vcsr_off[v0 + i + 1];
                for (int k = P.vcsr_off[v0 + i]; k < k1; k++) {
                    const uint32_t q = P.vcsr[k];
                    sum += sflux[3 * (q >> 2) + (q & 3u)];
                }
                inv = P.inv_av[v0 + i];
            }
            float e = seta[i] + sum * inv;
            if (EXTRA) {
                if (P.W) e -= dt * __ldg(P.W + v0 + i);
                if (P.eta_sum) P.eta_sum[v0 + i] += seta[i];
            }
            seta[i] = e;
            if (publish) st_relaxed_gpu_u64(xout + v0 + i, tag_out | __float_as_uint(e));
            bad |= !(fabsf(e) <= a.eta_bound);
        }
        if (bad) atomicOr(P.status, 1u);
        __syncthreads();
        if (!more) break;
    }
    __syncthreads();

    for (int i = threadIdx.x; i < nown; i += T) P.eta_out[v0 + i] = seta[i];
#pragma unroll
    for (int j = 0; j < SPT; j++) {
        const int i = threadIdx.x + j * T;
        if (i < ns) {
            P.U[s0 + i] = u[j];
            if (i < nown_s) {
                const int w = P.sv[s0 + i].w;
                P.Umean[w] = make_float2((shi[j].x + slo[j].x) * a.inv_M, (shi[j].y + slo[j].y) * a.inv_M);
            }
        }
    }
    // the last block of the pack to leave (every block has read the base by then) sets
    // the next launch's base
    if (threadIdx.x == 0 && atomicAdd(exit_count, 1u) == gridDim.x - 1) {
        *exit_count = 0u;
        *base_word = base + (unsigned)P.M + 1u;
    }
}

// ---------------------------------------------------------------------------------
// The SESM substep (AB3-AM4, Eqs. 4.7-4.8) in the persistent form: one launch runs the
// M + 1 element passes and M vertex passes of a baroclinic step. Substep m (m >= 1)
// completes the momentum update
//     U^m = U^{m-1} + dt ( -f e_z x U_AB^{m-1} - g H_AM grad(eta_AM^m) + R ),
//     eta_AM^m = am0 eta^m + am1 eta^{m-1} + am2 eta^{m-2} + am3 eta^{m-3},
// then (m < M) forms U_AB^m = ab0 U^m + ab1 U^{m-1} + ab2 U^{m-2}, adds it to the
// compensated sum and updates eta^{m+1} = eta^m - dt (div(U_AB^m) + W). Levels before the
// start of the subcycle are level 0. A slot keeps U^{m-1}, U^{m-2}, U_AB^{m-1} and its sum
// in registers; a vertex keeps eta^m, eta^{m-1}, eta^{m-2} in the registers of the thread
// that updates it. The element pass needs only eta_AM at the corners, so the owner of a
// vertex forms eta_AM^{m+1} right after eta^{m+1} and exchanges that one value, with the
// same tagged words as the SE kernel (tag base + m for substep m, m = 1 .. M).
constexpr int kSesmThreads = 384;   // registers: 65536 / (2 x 384) = 85 per thread
constexpr int kSesmVpt = 2;         // own vertices per thread at most

template <int SPT, int NONLIN>
__global__ void __launch_bounds__(kSesmThreads, 2) k_persistent_sesm(PArgs P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_abort;
    const int p = P.pack_patch[P.pack_base + blockIdx.x];
    const int T = blockDim.x;
    const int s0 = P.patch_slot[p], ns = P.patch_slot[p + 1] - s0;
    const int nown_s = P.patch_own[p], nint = P.patch_int[p];
    const int v0 = P.patch_v[p], nown = P.patch_v[p + 1] - v0;
    const int hb = P.patch_halo[p], nhalo = P.patch_halo[p + 1] - hb;
    const int c0 = P.vcsr_off[v0], ncsr = P.vcsr_off[v0 + nown] - c0;
    const StepArgs a = P.a;
    const float dt = P.patch_dt[p];
    unsigned *base_word = P.flags + (size_t)(1 + 2 * P.pack_index) * kFlagStride;
    unsigned *exit_count = base_word + kFlagStride;
    const unsigned base = ld_relaxed_gpu(base_word);
    const unsigned abort_val = base + 1u == 0u ? 1u : base + 1u;   // never 0, unique per launch

    float *sem = reinterpret_cast<float *>(smem_raw);   // eta_AM of the own vertices
    float *sflux = reinterpret_cast<float *>(smem_raw + P.off_flux);
    float4 *s_g = reinterpret_cast<float4 *>(smem_raw + P.off_g);
    float4 *s_c = reinterpret_cast<float4 *>(smem_raw + P.off_c);
    float2 *s_r = reinterpret_cast<float2 *>(smem_raw + P.off_r);
    ushort4 *s_l = reinterpret_cast<ushort4 *>(smem_raw + P.off_l);
    unsigned short *s_off = reinterpret_cast<unsigned short *>(smem_raw + P.off_off);
    unsigned short *s_csr = reinterpret_cast<unsigned short *>(smem_raw + P.off_csr);
    float *s_inv = reinterpret_cast<float *>(smem_raw + P.off_inv);
    int *s_halo = reinterpret_cast<int *>(smem_raw + P.off_halo);

    for (int i = threadIdx.x; i < ns; i += T) {
        s_g[i] = P.sg[s0 + i];
        s_c[i] = P.sc[s0 + i];
        s_r[i] = P.R[s0 + i];
        s_l[i] = P.sl[s0 + i];
    }
    for (int i = threadIdx.x; i <= nown; i += T) s_off[i] = (unsigned short)(P.vcsr_off[v0 + i] - c0);
    for (int k = threadIdx.x; k < ncsr; k += T) {
        const uint32_t q = P.vcsr[c0 + k];
        s_csr[k] = (unsigned short)(3u * (q >> 2) + (q & 3u));
    }
    for (int i = threadIdx.x; i < nown; i += T) s_inv[i] = P.inv_av[v0 + i];
    for (int i = threadIdx.x; i < nhalo; i += T) s_halo[i] = P.halo_v[hb + i];
    if (threadIdx.x == 0) s_abort = 0;
    // slot state: U^{m-1}, U^{m-2}, U_AB^{m-1}, compensated sum; vertex state: eta^m,
    // eta^{m-1}, eta^{m-2}
    float2 u1[SPT], u2[SPT], uab[SPT], shi[SPT], slo[SPT];
#pragma unroll
    for (int j = 0; j < SPT; j++) {
        const int i = threadIdx.x + j * T;
        u1[j] = i < ns ? P.U[s0 + i] : make_float2(0.0f, 0.0f);
        u2[j] = u1[j];
        uab[j] = make_float2(0.0f, 0.0f);
        shi[j] = make_float2(0.0f, 0.0f);
        slo[j] = make_float2(0.0f, 0.0f);
    }
    float eh0[kSesmVpt], eh1[kSesmVpt], eh2[kSesmVpt];
#pragma unroll
    for (int k = 0; k < kSesmVpt; k++) {
        const int i = threadIdx.x + k * T;
        eh0[k] = i < nown ? P.eta_in[v0 + i] : 0.0f;
        eh1[k] = eh0[k];
        eh2[k] = eh0[k];
    }
    __syncthreads();

    // U_AB of a slot, its flux contributions and (owned slots) the compensated sum
    auto transport = [&](int j, int i, float2 u0, float2 ua, float2 ub, float4 g, float area) {
        const float fx = a.ab0 * u0.x + a.ab1 * ua.x + a.ab2 * ub.x;
        const float fy = a.ab0 * u0.y + a.ab1 * ua.y + a.ab2 * ub.y;
        if (i < nown_s) {
            two_sum_acc(shi[j].x, slo[j].x, fx);
            two_sum_acc(shi[j].y, slo[j].y, fy);
        }
        const float w = dt * area;
        const float q0 = w * (fx * g.x + fy * g.y);
        const float q1 = w * (fx * g.z + fy * g.w);
        sflux[3 * i + 0] = q0;
        sflux[3 * i + 1] = q1;
        sflux[3 * i + 2] = -(q0 + q1);
        uab[j] = make_float2(fx, fy);
    };
    // element pass of substep m >= 1 over the slots [lo, hi); corner eta_AM of own
    // vertices from shared memory, of halo vertices (with `xs` set) from the exchange
    bool ok = true;
    auto elements = [&](int lo, int hi, const unsigned long long *xs, unsigned tag, bool vertex) {
#pragma unroll
        for (int j = 0; j < SPT; j++) {
            const int i = threadIdx.x + j * T;
            if (i >= lo && i < hi) {
                const float4 g = s_g[i], c = s_c[i];
                const float2 r = s_r[i];
                const ushort4 l = s_l[i];
                float e0, e1, e2;
                if (xs) {
                    const int h0 = l.x < nown ? -1 : s_halo[l.x - nown], h1 = l.y < nown ? -1 : s_halo[l.y - nown],
                              h2 = l.z < nown ? -1 : s_halo[l.z - nown];
                    const unsigned long long w0 = h0 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h0);
                    const unsigned long long w1 = h1 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h1);
                    const unsigned long long w2 = h2 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h2);
                    e0 = h0 < 0 ? sem[l.x] : halo_eta(P, xs, h0, w0, tag, abort_val, ok);
                    e1 = h1 < 0 ? sem[l.y] : halo_eta(P, xs, h1, w1, tag, abort_val, ok);
                    e2 = h2 < 0 ? sem[l.z] : halo_eta(P, xs, h2, w2, tag, abort_val, ok);
                } else {
                    e0 = sem[l.x];
                    e1 = sem[l.y];
                    e2 = sem[l.z];
                }
                const float d0 = e0 - e2, d1 = e1 - e2;
                const float gx = d0 * g.x + d1 * g.z;
                const float gy = d0 * g.y + d1 * g.w;
                float H = c.y;
                if (NONLIN) H += (e0 + e1 + e2) * (1.0f / 3.0f);
                const float gH = a.g * H;
                // -f e_z x U_AB = (f U_AB_y, -f U_AB_x)
                float2 u0;
                u0.x = u1[j].x + dt * (c.z * uab[j].y - gH * gx + r.x);
                u0.y = u1[j].y + dt * (-c.z * uab[j].x - gH * gy + r.y);
                if (vertex) transport(j, i, u0, u1[j], u2[j], g, c.x);
                u2[j] = u1[j];
                u1[j] = u0;
            }
        }
    };

    const int npre = nint >= T ? (nint / T) * T : nint;
    for (int m = 0; m <= P.M; m++) {
        const bool vertex = m < P.M;
        if (m == 0) {
            // no momentum update: U_AB^0 from level 0 and its aliases
#pragma unroll
            for (int j = 0; j < SPT; j++) {
                const int i = threadIdx.x + j * T;
                if (i < ns) transport(j, i, u1[j], u1[j], u1[j], s_g[i], s_c[i].x);
            }
        } else {
            const unsigned tag = base + (unsigned)m;
            elements(0, npre, nullptr, 0u, vertex);
            elements(npre, ns, P.xb[m & 1], tag, vertex);
            if (!ok) s_abort = 1;
        }
        if (!vertex) break;
        __syncthreads();
        if (s_abort) break;

        // vertex pass: eta^{m+1}, then eta_AM^{m+1} for the own slots and the neighbours
        unsigned long long *xout = P.xb[(m + 1) & 1];
        const unsigned long long tag_out = (unsigned long long)(base + (unsigned)(m + 1)) << 32;
        const bool publish = p != a.silent_patch;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < kSesmVpt; k++) {
            const int i = threadIdx.x + k * T;
            if (i < nown) {
                float sum = 0.0f;
                const int k1 = s_off[i + 1];
                for (int q = s_off[i]; q < k1; q++) sum += sflux[s_csr[q]];
                float e = eh0[k] + sum * s_inv[i];
                if (P.W) e -= dt * __ldg(P.W + v0 + i);
                const float em = a.am0 * e + a.am1 * eh0[k] + a.am2 * eh1[k] + a.am3 * eh2[k];
                eh2[k] = eh1[k];
                eh1[k] = eh0[k];
                eh0[k] = e;
                sem[i] = em;
                if (publish) st_relaxed_gpu_u64(xout + v0 + i, tag_out | __float_as_uint(em));
                bad |= !(fabsf(e) <= a.eta_bound);
            }
        }
        if (bad) atomicOr(P.status, 1u);
        __syncthreads();
    }
    __syncthreads();

#pragma unroll
    for (int k = 0; k < kSesmVpt; k++) {
        const int i = threadIdx.x + k * T;
        if (i < nown) P.eta_out[v0 + i] = eh0[k];
    }
#pragma unroll
    for (int j = 0; j < SPT; j++) {
        const int i = threadIdx.x + j * T;
        if (i < ns) {
            P.U[s0 + i] = u1[j];
            if (i < nown_s) {
                const int w = P.sv[s0 + i].w;
                P.Umean[w] = make_float2((shi[j].x + slo[j].x) * a.inv_M, (shi[j].y + slo[j].y) * a.inv_M);
            }
        }
    }
    if (threadIdx.x == 0 && atomicAdd(exit_count, 1u) == gridDim.x - 1) {
        *exit_count = 0u;
        *base_word = base + (unsigned)P.M + 1u;
    }
}

void *sesm_kernel(int spt, int nonlin)
{
    switch (spt) {
    case 1: return nonlin ? (void *)k_persistent_sesm<1, 1> : (void *)k_persistent_sesm<1, 0>;
    case 2: return nonlin ? (void *)k_persistent_sesm<2, 1> : (void *)k_persistent_sesm<2, 0>;
    case 3: return nonlin ? (void *)k_persistent_sesm<3, 1> : (void *)k_persistent_sesm<3, 0>;
    case 4: return nonlin ? (void *)k_persistent_sesm<4, 1> : (void *)k_persistent_sesm<4, 0>;
    default: return nullptr;
    }
}

// extra: the freshwater flux or the step-mean elevation is set
template <int SPT, int CACHED>
void *persistent_fn(int nonlin, int extra)
{
    if (extra) return nonlin ? (void *)k_persistent<SPT, 1, CACHED, 1> : (void *)k_persistent<SPT, 0, CACHED, 1>;
    return nonlin ? (void *)k_persistent<SPT, 1, CACHED, 0> : (void *)k_persistent<SPT, 0, CACHED, 0>;
}

void *persistent_kernel(int spt, int nonlin, int cached, int extra)
{
    if (cached) {
        switch (spt) {
        case 1: return persistent_fn<1, 1>(nonlin, extra);
        case 2: return persistent_fn<2, 1>(nonlin, extra);
        case 3: return persistent_fn<3, 1>(nonlin, extra);
        case 4: return persistent_fn<4, 1>(nonlin, extra);
        default: return nullptr;
        }
    }
    switch (spt) {
    case 1: return persistent_fn<1, 0>(nonlin, extra);
    case 2: return persistent_fn<2, 0>(nonlin, extra);
    case 3: return persistent_fn<3, 0>(nonlin, extra);
    case 4: return persistent_fn<4, 0>(nonlin, extra);
    case 6: return persistent_fn<6, 0>(nonlin, extra);
    case 8: return persistent_fn<8, 0>(nonlin, extra);
    default: return nullptr;
    }
}

size_t flag_bytes(int npatch) { return sizeof(unsigned) * (2 * (size_t)npatch + 1) * kFlagStride; }

struct SmemLayout {
    int off_flux, off_g, off_c, off_r, off_l, off_off, off_csr, off_inv, off_halo;
    size_t total_plain, total_cached;
};

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

SmemLayout smem_layout(const PatchMax &m)
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

}  // namespace

size_t persistent_flag_bytes(int npatch) { return flag_bytes(npatch); }

PersistentPlan persistent_plan(const PatchMax &m, int blocks_per_sm)
{
    PersistentPlan plan;
    int dev = 0, smem_optin = 0, smem_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return plan;
    }
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    const int max_threads = 1024 / blocks_per_sm;
    // fewest slots per thread such that one block of at most max_threads covers the
    // largest patch; the block is then sized to that patch (multiple of 32)
    static const int spts[] = {1, 2, 3, 4, 6, 8};
    int spt = 0, t = 0;
    for (int cand : spts) {
        const int need = (m.slots + cand - 1) / cand;
        const int tt = ((need + 31) / 32) * 32;
        if (tt <= max_threads) {
            spt = cand;
            t = tt < 32 ? 32 : tt;
            break;
        }
    }
    if (!spt) return plan;
    const SmemLayout L = smem_layout(m);
    // per block: the opt-in limit, and the SM's capacity shared by blocks_per_sm blocks
    // (1 KB of each block's share is reserved by the system, plus the kernel's static shared)
    size_t budget = (size_t)smem_optin - 1024;
    const size_t share = (size_t)smem_sm / (size_t)blocks_per_sm;
    if (share < 2048) return plan;
    budget = std::min(budget, share - 2048);
    // the cached variant indexes incidence entries and offsets with 16 bits
    int cached = (spt <= 4 && L.total_cached <= budget && m.csr < 65536 && m.slots < 16384) ? 1 : 0;
    const size_t smem = cached ? L.total_cached : L.total_plain;
    if (smem > budget) return plan;
    // every variant the plan may launch must reach blocks_per_sm resident blocks
    for (int nonlin = 0; nonlin < 2; nonlin++)
        for (int extra = 0; extra < 2; extra++) {
            void *fn = persistent_kernel(spt, nonlin, cached, extra);
            int occ = 0;
            if (!fn || raise_smem_limit(fn) < (int)smem ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, t, smem) != cudaSuccess ||
                occ < blocks_per_sm) {
                cudaGetLastError();
                return plan;
            }
        }
    plan.slots_per_thread = spt;
    plan.threads = t;
    plan.cached = cached;
    plan.smem = smem;
    return plan;
}

cudaError_t persistent_prepare(const PersistentPlan &plan)
{
    for (int nonlin = 0; nonlin < 2; nonlin++)
        for (int extra = 0; extra < 2; extra++) {
            void *fn = persistent_kernel(plan.slots_per_thread, nonlin, plan.cached, extra);
            if (!fn || raise_smem_limit(fn) < (int)plan.smem) return cudaErrorInvalidValue;
        }
    return cudaSuccess;
}

namespace {

PArgs make_pargs(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity, const PatchMax &mx)
{
    PArgs P;
    P.patch_slot = m.patch_slot;
    P.patch_own = m.patch_own;
    P.patch_int = m.patch_int;
    P.patch_v = m.patch_v;
    P.patch_halo = m.patch_halo;
    P.halo_v = m.halo_v;
    P.patch_nbr = m.patch_nbr;
    P.nbr = m.nbr;
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

// One cooperative launch per pack, with the pack's own plan and shared-memory layout;
// all packs of a step use the same elevation parity, and each pack has its own tag base
// (the exchange buffers need no clearing).
template <class Kernel>
cudaError_t launch_packs(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity,
                         const std::vector<PackPlan> &packs, bool sesm, Kernel kernel, cudaStream_t stream)
{
    for (size_t k = 0; k < packs.size(); k++) {
        const PackPlan &pk = packs[k];
        const PersistentPlan &plan = sesm ? pk.plan_sesm : pk.plan;
        void *fn = kernel(plan);
        if (!fn) return cudaErrorInvalidValue;
        PArgs P = make_pargs(m, s, a, M, parity, pk.mx);
        P.pack_base = pk.base;
        P.pack_index = (int)k;
        void *args[] = {&P};
        cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(pk.nblocks), dim3(plan.threads), args, plan.smem, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_persistent(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity,
                              const std::vector<PackPlan> &packs, cudaStream_t stream)
{
    const int extra = s.W != nullptr || s.eta_sum != nullptr;
    return launch_packs(m, s, a, M, parity, packs, false,
                        [&](const PersistentPlan &p) {
                            return persistent_kernel(p.slots_per_thread, a.nonlinear_h, p.cached, extra);
                        },
                        stream);
}

PersistentPlan persistent_plan_sesm(const PatchMax &m, int blocks_per_sm)
{
    PersistentPlan plan;
    int dev = 0, smem_optin = 0, smem_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return plan;
    }
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    // fewest slots per thread such that one block of at most kSesmThreads covers the
    // largest patch, whose own vertices must then fit kSesmVpt per thread
    int spt = 0, t = 0;
    for (int cand = 1; cand <= 4; cand++) {
        const int need = (m.slots + cand - 1) / cand;
        const int tt = std::max(32, ((need + 31) / 32) * 32);
        if (tt <= kSesmThreads) {
            spt = cand;
            t = tt;
            break;
        }
    }
    if (!spt || m.vertices > kSesmVpt * t) return plan;
    const SmemLayout L = smem_layout(m);
    size_t budget = (size_t)smem_optin - 1024;
    const size_t share = (size_t)smem_sm / (size_t)blocks_per_sm;
    if (share < 2048) return plan;
    budget = std::min(budget, share - 2048);
    if (L.total_cached > budget || m.csr >= 65536 || m.slots >= 16384) return plan;
    for (int nonlin = 0; nonlin < 2; nonlin++) {
        void *fn = sesm_kernel(spt, nonlin);
        int occ = 0;
        if (!fn || raise_smem_limit(fn) < (int)L.total_cached ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, t, L.total_cached) != cudaSuccess ||
            occ < blocks_per_sm) {
            cudaGetLastError();
            return plan;
        }
    }
    plan.slots_per_thread = spt;
    plan.threads = t;
    plan.cached = 1;
    plan.blocks_per_sm = blocks_per_sm;
    plan.smem = L.total_cached;
    return plan;
}

cudaError_t persistent_prepare_sesm(const PersistentPlan &plan)
{
    for (int nonlin = 0; nonlin < 2; nonlin++) {
        void *fn = sesm_kernel(plan.slots_per_thread, nonlin);
        if (!fn || raise_smem_limit(fn) < (int)plan.smem) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_persistent_sesm(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity,
                                   const std::vector<PackPlan> &packs, cudaStream_t stream)
{
    return launch_packs(m, s, a, M, parity, packs, true,
                        [&](const PersistentPlan &p) { return sesm_kernel(p.slots_per_thread, a.nonlinear_h); },
                        stream);
}

}  // namespace sesw
