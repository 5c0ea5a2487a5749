// The persistent step kernel of libsesw (sm_103a): one cooperative launch runs all M
// substeps of Eq. (4.10) of a baroclinic step, with the time-mean transport of Eq.
// (4.12) and the freshwater flux of Eq. (4.5).
#include "sesw_persistent.cuh"

namespace sesw {

namespace {

// ---------------------------------------------------------------------------------
// Persistent kernel: one launch per baroclinic step, one block per patch, all blocks
// resident (cooperative launch). A block keeps the elevation of its own and halo
// vertices and the per-corner fluxes in shared memory, and the transport and the
// compensated flux sum of its slots in registers, for all M substeps. When it fits
// (CACHED = 1), the patch's static slot data, incidence lists, 1/A_v and halo index list
// are also copied to shared memory once per step; with CACHED = 2 (patches whose static slot
// data do not fit) only the incidences, 1/A_v and the halo index list.
//
// Substep m: update the interior slots (corners all own vertices); update the other
// slots, reading the halo elevation from the exchange buffer of parity m; vertex pass;
// write the own vertices' new elevation to the exchange buffer of parity m+1 (the
// exchange protocol is described in sesw_persistent.cuh). In the cached forms one thread
// per halo vertex fetches the halo elevation into shared memory during the interior rounds.
//
// Vertex order. Mesh preparation puts the vertices that other patches read first in
// each patch, so the vertex pass publishes them in its first round; where a patch has more
// halo vertices than threads, the halo words of a thread's last-round slot are requested
// right after its first element round and have usually arrived by the time the slot is
// updated.
//
// The slots' step coefficients come from DevMesh::slot_k (formed once per parameter change);
// with CACHED = 2 the low parts of the compensated sums live in shared memory.

// Element update of one slot (Eq. 4.10, first row, and the theta-weighted flux);
// coef = (dt A_e, g H0_e, f dt / 2, 1 / (1 + (f dt / 2)^2)).
// Packed FP32 pairs in the element update of the cached kernels (UNCACHED: kUncachedPacked).
constexpr int kUncachedPacked = 0;
// Cached kernels (CACHED = 1 or 2, the halo ids in shared memory): each substep, one thread per
// halo vertex requests its tagged word before the interior rounds and stores its value to
// shared memory after them, and every other slot then reads its corners from shared memory
// (one extra block barrier per substep; patches with more halo vertices than threads keep the
// per-slot halo reads).
constexpr int kHaloPrefetch = 1;

template <int NONLIN, int PACKED>
__device__ __forceinline__ void element_update(const float e0, const float e1, const float e2, const float4 g,
                                               const float4 coef, const float2 r, float2 &u, float2 &shi,
                                               float2 &slo, bool owned, float *flux3, float theta,
                                               float one_p_theta, float dt, float gconst)
{
    const float2 F =
        se_transport<NONLIN, PACKED>(e0, e1, e2, g, coef.y, gconst, coef.z, coef.w, dt, r, one_p_theta, theta, u);
    if (owned) two_sum_acc2<PACKED>(shi, slo, F);
    corner_fluxes<PACKED>(F, g, coef.x, flux3);
}

__device__ __forceinline__ float4 slot_coef(const float4 c, float g, float dt)
{
    const float aa = __fmul_rn(c.z, __fmul_rn(0.5f, dt));
    return make_float4(__fmul_rn(dt, c.x), __fmul_rn(g, c.y), aa, __frcp_rn(__fmaf_rn(aa, aa, 1.0f)));
}

// The step coefficients of every slot, once per parameter change: the persistent kernels
// read them instead of forming them each substep (or in each launch's prologue).
__global__ void k_slot_coef(int npatch, const int *__restrict__ patch_slot, const float *__restrict__ patch_dt,
                            const float4 *__restrict__ sc, float g, float4 *__restrict__ sk)
{
    for (int p = blockIdx.x; p < npatch; p += gridDim.x) {
        const float dt = patch_dt[p];
        for (int s = patch_slot[p] + threadIdx.x; s < patch_slot[p + 1]; s += blockDim.x) sk[s] = slot_coef(sc[s], g, dt);
    }
}

// EXTRA: the optional per-vertex terms (freshwater flux, step-mean elevation) may be set;
// the instantiation without them carries neither load nor branch.
// One baroclinic step of patch p, the block's patch in pack `pack` (npb blocks take part).
template <int SPT, int NONLIN, int CACHED, int EXTRA>
__device__ __forceinline__ void persistent_patch(const PArgs &P, const int p, const int pack, const int npb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_abort;
    const int T = blockDim.x;
    const int s0 = P.patch_slot[p], ns = P.patch_slot[p + 1] - s0;
    const int nown_s = P.patch_own[p], nint = P.patch_int[p];
    const int v0 = P.patch_v[p], nown = P.patch_v[p + 1] - v0;
    const int hb = P.patch_halo[p], nhalo = P.patch_halo[p + 1] - hb;
    const StepArgs a = P.a;
    const float dt = P.patch_dt[p];
    unsigned *base_word = P.flags + (size_t)(1 + 2 * pack) * kFlagStride;
    unsigned *exit_count = base_word + kFlagStride;
    const unsigned base = ld_relaxed_gpu(base_word);
    const unsigned abort_val = base + 1u == 0u ? 1u : base + 1u;   // never 0, unique per launch

    float *seta = reinterpret_cast<float *>(smem_raw);
    float *sflux = reinterpret_cast<float *>(smem_raw + P.off_flux);
    float4 *s_g = reinterpret_cast<float4 *>(smem_raw + P.off_g);
    float4 *s_c = reinterpret_cast<float4 *>(smem_raw + P.off_c);
    float2 *s_r = reinterpret_cast<float2 *>(smem_raw + P.off_r);
    ushort4 *s_l = reinterpret_cast<ushort4 *>(smem_raw + P.off_l);
    float *s_inv = reinterpret_cast<float *>(smem_raw + P.off_inv);
    int *s_halo = reinterpret_cast<int *>(smem_raw + P.off_halo);

    for (int i = threadIdx.x; i < nown; i += T) seta[i] = P.eta_in[v0 + i];
    for (int i = threadIdx.x; i < nhalo; i += T) seta[nown + i] = P.eta_in[P.halo_v[hb + i]];
    if (CACHED == 1) {
        for (int i = threadIdx.x; i < ns; i += T) {
            s_g[i] = P.sg[s0 + i];
            s_c[i] = P.sk[s0 + i];
            s_r[i] = P.R[s0 + i];
            s_l[i] = P.sl[s0 + i];
        }
    }
    if (CACHED) {
        cache_incidences(P, smem_raw, v0, nown);
        for (int i = threadIdx.x; i < nown; i += T) s_inv[i] = P.inv_av[v0 + i];
        for (int i = threadIdx.x; i < nhalo; i += T) s_halo[i] = P.halo_v[hb + i];
    }
    if (threadIdx.x == 0) s_abort = 0;
    // CACHED == 2: the low parts of the compensated sums live in shared memory (in the place
    // of the static slot data, which this form does not cache), to spare registers
    float2 *s_slo = reinterpret_cast<float2 *>(smem_raw + P.off_g);
    float2 u[SPT], shi[SPT], slo[SPT];
#pragma unroll
    for (int j = 0; j < SPT; j++) {
        const int i = threadIdx.x + j * T;
        u[j] = i < ns ? P.U[s0 + i] : make_float2(0.0f, 0.0f);
        shi[j] = make_float2(0.0f, 0.0f);
        slo[j] = make_float2(0.0f, 0.0f);
        if (CACHED == 2 && i < ns) s_slo[i] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();

    const float one_p_theta = __fadd_rn(1.0f, a.theta);
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
                if (CACHED == 1) {
                    g = s_g[i];
                    coef = s_c[i];
                    r = s_r[i];
                    l = s_l[i];
                } else {
                    g = P.sg[s0 + i];
                    coef = P.sk[s0 + i];
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
                element_update<NONLIN, CACHED == 1 ? 1 : kUncachedPacked>(e0, e1, e2, g, coef, r, u[j], shi[j],
                                       CACHED == 2 ? s_slo[i] : slo[j], i < nown_s, sflux + 3 * i,
                                       a.theta, one_p_theta, dt, a.g);
            }
        }
    };

    // element update of slot i (round j of this thread) from its corner elevations; the
    // round's registers are selected by comparison (j is a constant once unrolled)
    auto slot_update = [&](int j, int i, float e0, float e1, float e2) {
        float4 g, coef;
        float2 r;
        if (CACHED == 1) {
            g = s_g[i];
            coef = s_c[i];
            r = s_r[i];
        } else {
            g = P.sg[s0 + i];
            coef = P.sk[s0 + i];
            r = P.R[s0 + i];
        }
        float2 uu = u[0], sh = shi[0], sl = slo[0];
#pragma unroll
        for (int q = 1; q < SPT; q++)
            if (q == j) { uu = u[q]; sh = shi[q]; sl = slo[q]; }
        if (CACHED == 2) sl = s_slo[i];
        element_update<NONLIN, CACHED == 1 ? 1 : kUncachedPacked>(e0, e1, e2, g, coef, r, uu, sh, sl, i < nown_s, sflux + 3 * i, a.theta,
                               one_p_theta, dt, a.g);
#pragma unroll
        for (int q = 0; q < SPT; q++)
            if (q == j) { u[q] = uu; shi[q] = sh; slo[q] = sl; }
        if (CACHED == 2) s_slo[i] = sl;
    };

    // Slots updated first: whole rounds of interior slots (one per thread each), so that
    // no thread does more rounds in total than ceil(ns / T); the interior slots left over
    // go with the boundary slots, whose halo reads may have to wait for a neighbour.
    const int npre = nint >= T ? (nint / T) * T : nint;
    const bool hpre = kHaloPrefetch && CACHED != 0 && nhalo <= T;
    for (int m = 0; m < P.M; m++) {
        if (hpre && m > 0) {
            // this thread's halo word is requested before the interior rounds and stored to
            // shared memory after them; the other slots follow a barrier
            const unsigned long long *xs = P.xb[m & 1];
            const int hv = (int)threadIdx.x < nhalo ? s_halo[threadIdx.x] : -1;
            const unsigned long long hw = hv >= 0 ? ld_relaxed_gpu_u64(xs + hv) : 0ull;
#pragma unroll
            for (int j = 0; j < SPT; j++) {
                const int i = threadIdx.x + j * T;
                if (i < npre) {
                    const ushort4 l = CACHED == 1 ? s_l[i] : P.sl[s0 + i];
                    slot_update(j, i, seta[l.x], seta[l.y], seta[l.z]);
                }
            }
            if (hv >= 0) seta[nown + threadIdx.x] = halo_eta(P, xs, hv, hw, base + (unsigned)m, abort_val, ok);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < SPT; j++) {
                const int i = threadIdx.x + j * T;
                if (i >= npre && i < ns) {
                    const ushort4 l = CACHED == 1 ? s_l[i] : P.sl[s0 + i];
                    slot_update(j, i, seta[l.x], seta[l.y], seta[l.z]);
                }
            }
        } else if (m == 0 || SPT == 1) {
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
                        const ushort4 l = CACHED == 1 ? s_l[i] : P.sl[s0 + i];
                        const int h0 = l.x < nown ? -1 : hid[l.x - nown], h1 = l.y < nown ? -1 : hid[l.y - nown],
                                  h2 = l.z < nown ? -1 : hid[l.z - nown];
                        const float e0 = h0 < 0 ? seta[l.x] : halo_eta(P, xs, h0, q0, base + (unsigned)m, abort_val, ok);
                        const float e1 = h1 < 0 ? seta[l.y] : halo_eta(P, xs, h1, q1, base + (unsigned)m, abort_val, ok);
                        const float e2 = h2 < 0 ? seta[l.z] : halo_eta(P, xs, h2, q2, base + (unsigned)m, abort_val, ok);
                        slot_update(j, i, e0, e1, e2);
                    } else if (i < npre) {
                        const ushort4 l = CACHED == 1 ? s_l[i] : P.sl[s0 + i];
                        slot_update(j, i, seta[l.x], seta[l.y], seta[l.z]);
                    }
                } else if (i < ns) {
                    const ushort4 l = CACHED == 1 ? s_l[i] : P.sl[s0 + i];
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
                    const ushort4 l = CACHED == 1 ? s_l[ilast] : P.sl[s0 + ilast];
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
                sum = cached_flux_sum(P, smem_raw, i);
                inv = s_inv[i];
            } else {
                const int k1 = P.vcsr_off[v0 + i + 1];
                for (int k = P.vcsr_off[v0 + i]; k < k1; k++) {
                    const uint32_t q = P.vcsr[k];
                    sum += sflux[3 * (q >> 2) + (q & 3u)];
                }
                inv = P.inv_av[v0 + i];
            }
            float e = vertex_eta(seta[i], sum, inv);
            if (EXTRA) {
                if (P.W) e = __fmaf_rn(-dt, __ldg(P.W + v0 + i), e);
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
                const float2 lo = CACHED == 2 ? s_slo[i] : slo[j];
                P.Umean[w] = make_float2((shi[j].x + lo.x) * a.inv_M, (shi[j].y + lo.y) * a.inv_M);
            }
        }
    }
    // the last block of the pack to leave (every block of the pack has read the base by
    // then) sets the base of the pack's next step
    if (threadIdx.x == 0 && atomicAdd(exit_count, 1u) == (unsigned)npb - 1u) {
        *exit_count = 0u;
        *base_word = base + (unsigned)P.M + 1u;
    }
}

// A launch runs packs [P.pack_first, P.pack_last) one after another: block b takes patch b of
// each pack that has more than b patches. Packs exchange nothing with each other (a pack holds
// whole basins), so a block goes on to its next pack as soon as it is done with the last
// one, while other blocks still finish theirs; every block of a pack is resident, so the
// waits of a pack always end.
template <int SPT, int NONLIN, int CACHED, int EXTRA>
__global__ void __launch_bounds__(1024, 1) k_persistent(PArgs P)
{
    for (int k = P.pack_first; k < P.pack_last; k++) {
        const int b0 = P.pack_off[k], npb = P.pack_off[k + 1] - b0;
        if ((int)blockIdx.x < npb) persistent_patch<SPT, NONLIN, CACHED, EXTRA>(P, P.pack_patch[b0 + blockIdx.x], k, npb);
        __syncthreads();   // the next pack reuses the shared memory
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
    if (cached == 1) {
        switch (spt) {
        case 1: return persistent_fn<1, 1>(nonlin, extra);
        case 2: return persistent_fn<2, 1>(nonlin, extra);
        case 3: return persistent_fn<3, 1>(nonlin, extra);
        case 4: return persistent_fn<4, 1>(nonlin, extra);
        default: return nullptr;
        }
    }
    if (cached == 2) {
        switch (spt) {
        case 4: return persistent_fn<4, 2>(nonlin, extra);
        case 6: return persistent_fn<6, 2>(nonlin, extra);
        case 7: return persistent_fn<7, 2>(nonlin, extra);
        case 8: return persistent_fn<8, 2>(nonlin, extra);
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
    const SmemLayout L = smem_layout(m);
    // per block: the opt-in limit, and the SM's capacity shared by blocks_per_sm blocks
    // (1 KB of each block's share is reserved by the system, plus the kernel's static shared)
    size_t budget = (size_t)smem_optin - 1024;
    const size_t share = (size_t)smem_sm / (size_t)blocks_per_sm;
    if (share < 2048) return plan;
    budget = std::min(budget, share - 2048);
    // 7 slots per thread exist only with the vertices' data in shared memory (cached = 2)
    const bool vcached_fits = m.csr < 65536 && 3 * (size_t)m.slots < 65536 &&
                              L.total_vcached + sizeof(float2) * (size_t)m.slots <= budget;
    static const int spts[] = {1, 2, 3, 4, 6, 7, 8};
    int spt = 0, t = 0;
    for (int cand : spts) {
        const int need = (m.slots + cand - 1) / cand;
        const int tt = ((need + 31) / 32) * 32;
        if (tt <= max_threads && (cand != 7 || vcached_fits)) {
            spt = cand;
            t = tt < 32 ? 32 : tt;
            break;
        }
    }
    if (!spt) return plan;
    // the cached variants index incidence entries and offsets with 16 bits; the slots' static
    // data join the vertices' data in shared memory when they fit (cached = 1), else only the
    // vertices' data (cached = 2, with 4 or more slots per thread)
    int cached = 0;
    if (m.csr < 65536 && 3 * (size_t)m.slots < 65536) {
        if (spt <= 4 && L.total_cached <= budget && m.slots < 16384)
            cached = 1;
        else if (spt >= 4 && L.total_vcached + sizeof(float2) * (size_t)m.slots <= budget &&
                 persistent_kernel(spt, 0, 2, 0))
            cached = 2;
    }
    // cached = 2 keeps the low parts of the slots' compensated sums where the static data would go
    const size_t smem = cached == 1   ? L.total_cached
                        : cached == 2 ? L.total_vcached + sizeof(float2) * (size_t)m.slots
                                      : L.total_plain;
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

cudaError_t launch_persistent(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity,
                              const std::vector<PackGroup> &groups, cudaStream_t stream)
{
    const int extra = s.W != nullptr || s.eta_sum != nullptr;
    for (const PackGroup &g : groups) {
        cudaError_t e;
        if (g.plan.stream) {
            e = launch_persistent_stream_group(m, s, a, M, parity, g, stream);
        } else {
            void *fn = persistent_kernel(g.plan.slots_per_thread, a.nonlinear_h, g.plan.cached, extra);
            if (!fn) return cudaErrorInvalidValue;
            PArgs P = make_pargs(m, s, a, M, parity, g.mx);
            P.pack_first = g.first;
            P.pack_last = g.last;
            void *args[] = {&P};
            e = cudaLaunchCooperativeKernel(fn, dim3(g.nblocks), dim3(g.plan.threads), args, g.plan.smem, stream);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_slot_coef(const DevMesh &m, float g, cudaStream_t stream)
{
    if (m.npatch <= 0) return cudaSuccess;
    k_slot_coef<<<std::min(m.npatch, 152 * 16), 256, 0, stream>>>(m.npatch, m.patch_slot, m.patch_dt, m.slot_c, g,
                                                                 m.slot_k);
    return cudaGetLastError();
}

}  // namespace sesw
