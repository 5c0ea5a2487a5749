// The streaming persistent step kernel of libsesw (sm_103a), for patches too large to keep
// their state on chip: one cooperative launch runs all M substeps of Eq. (4.10) of a
// baroclinic step, with the time-mean transport of Eq. (4.12) and the freshwater flux of
// Eq. (4.5), like k_persistent, but the transport, the compensated sum and the static
// slot data stay in global memory (L2-resident across the substeps) and are read and
// written slot by slot. The elevation of the patch's own and halo vertices, the
// per-corner fluxes and the slots' corner indices (loaded once per launch) live in shared
// memory. With no per-slot registers carried between
// substeps, a block holds any number of slots per thread without spilling, and every
// load of a slot depends only on the slot's index, so it costs one L2 round trip.
#include "sesw_persistent.cuh"

namespace sesw {

namespace {

constexpr int kStreamThreads = 1024;   // 64 registers per thread at any residency
constexpr int kStreamPacked = 0;       // packed FP32 pairs in the element update

struct SArgs {
    PArgs P;
    float2 *Shi, *Slo;
    int off_idx;    // IDX: shared-memory offset of the cached corner indices (ushort4 per slot)
    int vcache;     // 1: the vertices' data (1/A_v, halo ids, incidences) is in shared memory at
                    // P.off_inv, P.off_halo and P.off_off / P.off_csr
};

// Shared-memory layout of the streaming kernel: the plain part (elevation, corner fluxes, zero
// word), the slots' corner indices (idx), then, when vc, the vertices' data laid out like the
// register kernel's. Returns the total; fills the offsets into P when P is given.
size_t stream_layout(const PatchMax &m, int idx, int vc, PArgs *P)
{
    const SmemLayout L = smem_layout(m);
    size_t o = align16(L.total_plain) + (idx ? sizeof(ushort4) * (size_t)m.slots : 0);
    if (!vc) return o;
    o = align16(o);
    const size_t off_inv = o;
    o = align16(o + sizeof(float) * (size_t)m.vertices);
    const size_t off_halo = o;
    o = align16(o + sizeof(int) * (size_t)m.halo);
    const size_t off_off = o;
    const size_t off_csr = align16(o + sizeof(unsigned short) * ((size_t)m.vertices + 1));
    const size_t end = L.inc8 ? align16(o + sizeof(unsigned short) * kIncWidth * (size_t)m.vertices)
                              : align16(off_csr + sizeof(unsigned short) * (size_t)m.csr);
    if (P) {
        P->off_inv = (int)off_inv;
        P->off_halo = (int)off_halo;
        P->off_off = (int)off_off;
        P->off_csr = (int)off_csr;
    }
    return end;
}

// Element update of one slot (Eq. 4.10, first row, and the theta-weighted flux) from its
// corner elevations, with everything else read from and written back to global memory.
template <int NONLIN>
__device__ __forceinline__ void stream_slot(const SArgs &A, int s, int i, bool owned, bool first, float e0, float e1,
                                            float e2, float dt, float *sflux)
{
    const PArgs &P = A.P;
    const StepArgs &a = P.a;
    // c = (dt A_e, g H0_e, f dt / 2, 1 / (1 + (f dt / 2)^2)), formed once per parameter change
    const float4 g = __ldg(P.sg + s), c = __ldg(P.sk + s);
    const float2 r = __ldg(P.R + s);
    float2 u = P.U[s];
    float2 shi = make_float2(0.0f, 0.0f), slo = shi;
    if (owned && !first) {
        shi = A.Shi[s];
        slo = A.Slo[s];
    }
    const float2 F = se_transport<NONLIN, kStreamPacked>(e0, e1, e2, g, c.y, a.g, c.z, c.w, dt, r,
                                          __fadd_rn(1.0f, a.theta), a.theta, u);
    P.U[s] = u;
    if (owned) {
        two_sum_acc2<kStreamPacked>(shi, slo, F);
        A.Shi[s] = shi;
        A.Slo[s] = slo;
    }
    corner_fluxes<kStreamPacked>(F, g, c.x, sflux + 3 * i);
}

// EXTRA: the optional per-vertex terms (freshwater flux, step-mean elevation) may be set.
// IDX = 1 keeps the slots' corner indices in shared memory; IDX = 0 (patches too large for
// that) reads them from global memory every substep.
template <int NONLIN, int EXTRA, int IDX>
__device__ __forceinline__ void stream_patch(const SArgs &A, const int p, const int pack, const int npb)
{
    const PArgs &P = A.P;
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
    ushort4 *s_l = reinterpret_cast<ushort4 *>(smem_raw + A.off_idx);
    float *s_inv = reinterpret_cast<float *>(smem_raw + P.off_inv);
    int *s_halo = reinterpret_cast<int *>(smem_raw + P.off_halo);
    if (IDX)
        for (int i = threadIdx.x; i < ns; i += T) s_l[i] = __ldg(P.sl + s0 + i);
    for (int i = threadIdx.x; i < nown; i += T) seta[i] = P.eta_in[v0 + i];
    for (int i = threadIdx.x; i < nhalo; i += T) seta[nown + i] = P.eta_in[P.halo_v[hb + i]];
    if (A.vcache) {
        cache_incidences(P, smem_raw, v0, nown);
        for (int i = threadIdx.x; i < nown; i += T) s_inv[i] = P.inv_av[v0 + i];
        for (int i = threadIdx.x; i < nhalo; i += T) s_halo[i] = P.halo_v[hb + i];
    }
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();

    const int *hid = A.vcache ? s_halo : P.halo_v + hb;
    bool ok = true;
    for (int m = 0; m < P.M; m++) {
        const unsigned tag = base + (unsigned)m;
        const unsigned long long *xs = P.xb[m & 1];
        const bool first = m == 0;
        // interior slots (all corners own vertices) first, then the others, whose halo
        // reads may have to wait for a neighbour; every halo value is in shared memory
        // at m = 0
        const int nfirst = first ? ns : nint;
        // with the halo ids in shared memory, one thread per halo vertex requests its tagged
        // word now and stores its value to shared memory after the interior slots; the other
        // slots then read all corners from shared memory
        const bool hpre = !first && A.vcache && nhalo <= T;
        const int hv = hpre && (int)threadIdx.x < nhalo ? hid[threadIdx.x] : -1;
        const unsigned long long hw = hv >= 0 ? ld_relaxed_gpu_u64(xs + hv) : 0ull;
#pragma unroll 8
        for (int i = threadIdx.x; i < nfirst; i += T) {
            const ushort4 l = IDX ? s_l[i] : __ldg(P.sl + s0 + i);
            stream_slot<NONLIN>(A, s0 + i, i, i < nown_s, first, seta[l.x], seta[l.y], seta[l.z], dt, sflux);
        }
        if (hpre) {
            if (hv >= 0) seta[nown + threadIdx.x] = halo_eta(P, xs, hv, hw, tag, abort_val, ok);
            __syncthreads();
#pragma unroll 8
            for (int i = nfirst + threadIdx.x; i < ns; i += T) {
                const ushort4 l = IDX ? s_l[i] : __ldg(P.sl + s0 + i);
                stream_slot<NONLIN>(A, s0 + i, i, i < nown_s, false, seta[l.x], seta[l.y], seta[l.z], dt, sflux);
            }
        }
#pragma unroll 8
        for (int i = nfirst + threadIdx.x; !hpre && i < ns; i += T) {
            const ushort4 l = IDX ? s_l[i] : __ldg(P.sl + s0 + i);
            const int h0 = l.x < nown ? -1 : hid[l.x - nown], h1 = l.y < nown ? -1 : hid[l.y - nown],
                      h2 = l.z < nown ? -1 : hid[l.z - nown];
            const unsigned long long w0 = h0 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h0);
            const unsigned long long w1 = h1 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h1);
            const unsigned long long w2 = h2 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h2);
            const float e0 = h0 < 0 ? seta[l.x] : halo_eta(P, xs, h0, w0, tag, abort_val, ok);
            const float e1 = h1 < 0 ? seta[l.y] : halo_eta(P, xs, h1, w1, tag, abort_val, ok);
            const float e2 = h2 < 0 ? seta[l.z] : halo_eta(P, xs, h2, w2, tag, abort_val, ok);
            stream_slot<NONLIN>(A, s0 + i, i, i < nown_s, first, e0, e1, e2, dt, sflux);
        }
        if (!ok) s_abort = 1;
        __syncthreads();
        if (s_abort) break;

        // vertex pass; the new elevation of own vertices also goes to the exchange buffer
        const bool more = m + 1 < P.M;
        unsigned long long *xout = P.xb[(m + 1) & 1];
        const unsigned long long tag_out = (unsigned long long)(tag + 1u) << 32;
        const bool publish = more && p != a.silent_patch;
        bool bad = false;
        for (int i = threadIdx.x; i < nown; i += T) {
            float sum = 0.0f, inv;
            if (A.vcache) {
                sum = cached_flux_sum(P, smem_raw, i);
                inv = s_inv[i];
            } else {
                const int k1 = __ldg(P.vcsr_off + v0 + i + 1);
                for (int k = __ldg(P.vcsr_off + v0 + i); k < k1; k++) {
                    const uint32_t q = __ldg(P.vcsr + k);
                    sum += sflux[3 * (q >> 2) + (q & 3u)];
                }
                inv = __ldg(P.inv_av + v0 + i);
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
    for (int i = threadIdx.x; i < nown_s; i += T) {
        const int s = s0 + i;
        const int w = P.sv[s].w;
        const float2 hi = A.Shi[s], lo = A.Slo[s];
        P.Umean[w] = make_float2((hi.x + lo.x) * a.inv_M, (hi.y + lo.y) * a.inv_M);
    }
    // the last block of the pack to leave (every block of the pack has read the base by
    // then) sets the base of the pack's next step
    if (threadIdx.x == 0 && atomicAdd(exit_count, 1u) == (unsigned)npb - 1u) {
        *exit_count = 0u;
        *base_word = base + (unsigned)P.M + 1u;
    }
}

// The packs [P.pack_first, P.pack_last) one after another, as in k_persistent.
template <int NONLIN, int EXTRA, int IDX>
__global__ void __launch_bounds__(kStreamThreads, 1) k_persistent_stream(SArgs A)
{
    const PArgs &P = A.P;
    for (int k = P.pack_first; k < P.pack_last; k++) {
        const int b0 = P.pack_off[k], npb = P.pack_off[k + 1] - b0;
        if ((int)blockIdx.x < npb) stream_patch<NONLIN, EXTRA, IDX>(A, P.pack_patch[b0 + blockIdx.x], k, npb);
        __syncthreads();   // the next pack reuses the shared memory
    }
}

template <int IDX>
void *stream_kernel_of(int nonlin, int extra)
{
    if (extra) return nonlin ? (void *)k_persistent_stream<1, 1, IDX> : (void *)k_persistent_stream<0, 1, IDX>;
    return nonlin ? (void *)k_persistent_stream<1, 0, IDX> : (void *)k_persistent_stream<0, 0, IDX>;
}

void *stream_kernel(int nonlin, int extra, int idx)
{
    return idx ? stream_kernel_of<1>(nonlin, extra) : stream_kernel_of<0>(nonlin, extra);
}

}  // namespace

PersistentPlan persistent_plan_stream(const PatchMax &m, int blocks_per_sm, int idx_mode)
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
    // as many threads as the residency allows, but no more than the largest patch has slots
    const int t = std::min(std::min(kStreamThreads, 1024 / blocks_per_sm), std::max(32, ((m.slots + 31) / 32) * 32));
    const SmemLayout L = smem_layout(m);
    size_t budget = (size_t)smem_optin - 1024;
    const size_t share = (size_t)smem_sm / (size_t)blocks_per_sm;
    if (share < 2048) return plan;
    budget = std::min(budget, share - 2048);
    // the corner indices join the shared memory when they fit (idx_mode 0: never), and then the
    // vertices' data when it fits too (the cached incidences index the fluxes with 16 bits)
    int idx = 1;
    size_t need = stream_layout(m, 1, 0, nullptr);
    if (need > budget || idx_mode == 0) {
        idx = 0;
        need = L.total_plain;
    }
    if (need > budget) return plan;
    int vc = 0;
    if (m.csr < 65536 && 3 * (size_t)m.slots < 65536 && stream_layout(m, idx, 1, nullptr) <= budget) {
        vc = 1;
        need = stream_layout(m, idx, 1, nullptr);
    }
    for (int nonlin = 0; nonlin < 2; nonlin++)
        for (int extra = 0; extra < 2; extra++) {
            void *fn = stream_kernel(nonlin, extra, idx);
            int occ = 0;
            if (!fn || raise_smem_limit(fn) < (int)need ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, t, need) != cudaSuccess ||
                occ < blocks_per_sm) {
                cudaGetLastError();
                return plan;
            }
        }
    plan.slots_per_thread = (m.slots + t - 1) / t;   // rounds of the slot loop (not registers)
    plan.threads = t;
    plan.cached = vc;    // streaming kernels: 1 when the vertices' data is in shared memory
    plan.stream = idx ? 1 : 2;
    plan.blocks_per_sm = blocks_per_sm;
    plan.smem = need;
    return plan;
}

cudaError_t persistent_prepare_stream(const PersistentPlan &plan)
{
    for (int nonlin = 0; nonlin < 2; nonlin++)
        for (int extra = 0; extra < 2; extra++) {
            void *fn = stream_kernel(nonlin, extra, plan.stream == 1);
            if (!fn || raise_smem_limit(fn) < (int)plan.smem) return cudaErrorInvalidValue;
        }
    return cudaSuccess;
}

cudaError_t launch_persistent_stream_group(const DevMesh &m, const DevState &s, const StepArgs &a, int M, int parity,
                                           const PackGroup &g, cudaStream_t stream)
{
    SArgs A;
    A.P = make_pargs(m, s, a, M, parity, g.mx);
    A.P.pack_first = g.first;
    A.P.pack_last = g.last;
    A.Shi = s.S_hi;
    A.Slo = s.S_lo;
    A.off_idx = (int)align16(smem_layout(g.mx).total_plain);
    A.vcache = g.plan.cached;
    if (A.vcache) stream_layout(g.mx, g.plan.stream == 1, 1, &A.P);
    void *fn = stream_kernel(a.nonlinear_h, s.W != nullptr || s.eta_sum != nullptr, g.plan.stream == 1);
    if (!fn) return cudaErrorInvalidValue;
    void *args[] = {&A};
    return cudaLaunchCooperativeKernel(fn, dim3(g.nblocks), dim3(g.plan.threads), args, g.plan.smem, stream);
}

}  // namespace sesw
