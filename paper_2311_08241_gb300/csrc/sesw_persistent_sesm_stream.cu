// The streaming SESM step kernel of libsesw (sm_103a), for patches too large to keep the
// scheme's state on chip: one cooperative launch runs a baroclinic step of the AB3-AM4
// substep of Eqs. (4.7)-(4.8), like k_persistent_sesm, with the time-mean transport of
// Eq. (4.12) and the freshwater flux of Eq. (4.5). The transport levels U^{m-1} and
// U^{m-2}, the AB3 transport U_AB^{m-1}, the compensated sum and the static slot data
// stay in global memory (L2-resident across the substeps) and are read and written slot
// by slot; the AM4 elevation of the own and halo vertices, the corner fluxes, the
// three-level elevation history of the own vertices and the slots' corner indices (loaded
// once per launch) live in shared memory. The owner of
// a vertex exchanges its AM4 elevation as in k_persistent_sesm.
#include "sesw_persistent.cuh"

namespace sesw {

namespace {

constexpr int kSesmStreamThreads = 1024;   // 64 registers per thread at any residency

struct QArgs {
    PArgs P;
    float2 *U2, *UAB;     // per slot: U^{m-2} and U_AB^{m-1}
    float2 *Shi, *Slo;    // per slot: the compensated sum of the AB3 transports
    int off_hist;         // shared-memory offset of the elevation history (bytes)
    int off_idx;          // IDX: shared-memory offset of the cached corner indices (ushort4 per slot)
    int vmax;             // own vertices of the largest patch (stride of the history)
    int vcache;           // 1: the vertices' data (1/A_v, halo ids, incidences) is in shared memory
                          // at P.off_inv, P.off_halo and P.off_off / P.off_csr
};

// U_AB of slot s from its levels, its flux contributions and (owned) the compensated sum;
// `first` starts the sum.
__device__ __forceinline__ float2 sesm_transport(const QArgs &A, int s, int i, bool owned, bool first, float2 u0,
                                                 float2 ua, float2 ub, float4 g, float area, float dt, float *sflux)
{
    const StepArgs &a = A.P.a;
    const float2 F = sesm_ab3(u0, ua, ub, a.ab0, a.ab1, a.ab2);
    if (owned) {
        float2 hi = make_float2(0.0f, 0.0f), lo = hi;
        if (!first) {
            hi = A.Shi[s];
            lo = A.Slo[s];
        }
        two_sum_acc2(hi, lo, F);
        A.Shi[s] = hi;
        A.Slo[s] = lo;
    }
    corner_fluxes(F, g, __fmul_rn(dt, area), sflux + 3 * i);
    return F;
}

// Momentum update of slot s (substep m >= 1) from its corner eta_AM, then (vertex) its
// transport; the levels shift in global memory.
template <int NONLIN>
__device__ __forceinline__ void sesm_slot(const QArgs &A, int s, int i, bool owned, bool vertex, float e0, float e1,
                                          float e2, float dt, float *sflux)
{
    const PArgs &P = A.P;
    const StepArgs &a = P.a;
    const float4 g = __ldg(P.sg + s), c = __ldg(P.sc + s);
    const float2 r = __ldg(P.R + s);
    const float2 u1 = P.U[s], u2 = A.U2[s], uab = A.UAB[s];
    const float2 u0 = sesm_momentum<NONLIN>(e0, e1, e2, g, c.y, a.g, c.z, dt, r, u1, uab);
    if (vertex) {
        A.UAB[s] = sesm_transport(A, s, i, owned, false, u0, u1, u2, g, c.x, dt, sflux);
        A.U2[s] = u1;
    }
    P.U[s] = u0;
}

// IDX = 1 keeps the slots' corner indices in shared memory; IDX = 0 (patches too large for
// that) reads them from global memory every substep.
template <int NONLIN, int IDX>
__global__ void __launch_bounds__(kSesmStreamThreads, 1) k_persistent_sesm_stream(QArgs A)
{
    const PArgs &P = A.P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_abort;
    const int p = P.pack_patch[P.pack_base + blockIdx.x];
    const int T = blockDim.x;
    const int s0 = P.patch_slot[p], ns = P.patch_slot[p + 1] - s0;
    const int nown_s = P.patch_own[p], nint = P.patch_int[p];
    const int v0 = P.patch_v[p], nown = P.patch_v[p + 1] - v0;
    const StepArgs a = P.a;
    const float dt = P.patch_dt[p];
    unsigned *base_word = P.flags + (size_t)(1 + 2 * P.pack_index) * kFlagStride;
    unsigned *exit_count = base_word + kFlagStride;
    const unsigned base = ld_relaxed_gpu(base_word);
    const unsigned abort_val = base + 1u == 0u ? 1u : base + 1u;   // never 0, unique per launch

    float *sem = reinterpret_cast<float *>(smem_raw);   // eta_AM of own and halo vertices
    float *sflux = reinterpret_cast<float *>(smem_raw + P.off_flux);
    float *h0 = reinterpret_cast<float *>(smem_raw + A.off_hist);   // eta^m, eta^{m-1}, eta^{m-2} of own vertices
    float *h1 = h0 + A.vmax, *h2 = h1 + A.vmax;
    ushort4 *s_l = reinterpret_cast<ushort4 *>(smem_raw + A.off_idx);
    float *s_inv = reinterpret_cast<float *>(smem_raw + P.off_inv);
    int *s_halo = reinterpret_cast<int *>(smem_raw + P.off_halo);
    const int hb = P.patch_halo[p], nhalo = P.patch_halo[p + 1] - hb;
    if (IDX)
        for (int i = threadIdx.x; i < ns; i += T) s_l[i] = __ldg(P.sl + s0 + i);
    for (int i = threadIdx.x; i < nown; i += T) {
        const float x = __ldg(P.eta_in + v0 + i);
        h0[i] = x;
        h1[i] = x;
        h2[i] = x;
    }
    if (A.vcache) {
        cache_incidences(P, smem_raw, v0, nown);
        for (int i = threadIdx.x; i < nown; i += T) s_inv[i] = P.inv_av[v0 + i];
        for (int i = threadIdx.x; i < nhalo; i += T) s_halo[i] = P.halo_v[hb + i];
    }
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();

    const int *hid = A.vcache ? s_halo : P.halo_v + hb;
    bool ok = true;
    for (int m = 0; m <= P.M; m++) {
        const bool vertex = m < P.M;
        if (m == 0) {
            // no momentum update: U_AB^0 from level 0 and its aliases
#pragma unroll 8
            for (int i = threadIdx.x; i < ns; i += T) {
                const int s = s0 + i;
                const float2 u = P.U[s];
                A.UAB[s] = sesm_transport(A, s, i, i < nown_s, true, u, u, u, __ldg(P.sg + s), __ldg(P.sc + s).x, dt,
                                          sflux);
                A.U2[s] = u;
            }
        } else {
            const unsigned tag = base + (unsigned)m;
            const unsigned long long *xs = P.xb[m & 1];
#pragma unroll 8
            for (int i = threadIdx.x; i < nint; i += T) {
                const ushort4 l = IDX ? s_l[i] : __ldg(P.sl + s0 + i);
                sesm_slot<NONLIN>(A, s0 + i, i, i < nown_s, vertex, sem[l.x], sem[l.y], sem[l.z], dt, sflux);
            }
#pragma unroll 8
            for (int i = nint + threadIdx.x; i < ns; i += T) {
                const ushort4 l = IDX ? s_l[i] : __ldg(P.sl + s0 + i);
                const int q0 = l.x < nown ? -1 : hid[l.x - nown], q1 = l.y < nown ? -1 : hid[l.y - nown],
                          q2 = l.z < nown ? -1 : hid[l.z - nown];
                const unsigned long long w0 = q0 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + q0);
                const unsigned long long w1 = q1 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + q1);
                const unsigned long long w2 = q2 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + q2);
                const float e0 = q0 < 0 ? sem[l.x] : halo_eta(P, xs, q0, w0, tag, abort_val, ok);
                const float e1 = q1 < 0 ? sem[l.y] : halo_eta(P, xs, q1, w1, tag, abort_val, ok);
                const float e2 = q2 < 0 ? sem[l.z] : halo_eta(P, xs, q2, w2, tag, abort_val, ok);
                sesm_slot<NONLIN>(A, s0 + i, i, i < nown_s, vertex, e0, e1, e2, dt, sflux);
            }
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
            float e = vertex_eta(h0[i], sum, inv);
            if (P.W) e = __fmaf_rn(-dt, __ldg(P.W + v0 + i), e);
            const float em = sesm_am4(e, h0[i], h1[i], h2[i], a.am0, a.am1, a.am2, a.am3);
            h2[i] = h1[i];
            h1[i] = h0[i];
            h0[i] = e;
            sem[i] = em;
            if (publish) st_relaxed_gpu_u64(xout + v0 + i, tag_out | __float_as_uint(em));
            bad |= !(fabsf(e) <= a.eta_bound);
        }
        if (bad) atomicOr(P.status, 1u);
        __syncthreads();
    }
    __syncthreads();

    for (int i = threadIdx.x; i < nown; i += T) P.eta_out[v0 + i] = h0[i];
    for (int i = threadIdx.x; i < nown_s; i += T) {
        const int s = s0 + i;
        const int w = P.sv[s].w;
        const float2 hi = A.Shi[s], lo = A.Slo[s];
        P.Umean[w] = make_float2((hi.x + lo.x) * a.inv_M, (hi.y + lo.y) * a.inv_M);
    }
    // the last block of the pack to leave (every block has read the base by then) sets
    // the next launch's base
    if (threadIdx.x == 0 && atomicAdd(exit_count, 1u) == gridDim.x - 1) {
        *exit_count = 0u;
        *base_word = base + (unsigned)P.M + 1u;
    }
}

void *sesm_stream_kernel(int nonlin, int idx)
{
    if (idx) return nonlin ? (void *)k_persistent_sesm_stream<1, 1> : (void *)k_persistent_sesm_stream<0, 1>;
    return nonlin ? (void *)k_persistent_sesm_stream<1, 0> : (void *)k_persistent_sesm_stream<0, 0>;
}

size_t hist_offset(const SmemLayout &L) { return align16(L.total_plain); }

size_t idx_offset(const PatchMax &m) { return hist_offset(smem_layout(m)) + align16(3 * sizeof(float) * (size_t)m.vertices); }

// Shared memory of the SESM streaming kernel: the plain part, the elevation history, the
// corner indices (idx), then, when vc, the vertices' data laid out like the register kernel's
// (offsets into P when P is given).
size_t sesm_stream_smem(const PatchMax &m, int idx, int vc = 0, PArgs *P = nullptr)
{
    size_t o = idx ? idx_offset(m) + sizeof(ushort4) * (size_t)m.slots : idx_offset(m);
    if (!vc) return o;
    const SmemLayout L = smem_layout(m);
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

}  // namespace

PersistentPlan persistent_plan_sesm_stream(const PatchMax &m, int blocks_per_sm, int idx_mode)
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
    const int t =
        std::min(std::min(kSesmStreamThreads, 1024 / blocks_per_sm), std::max(32, ((m.slots + 31) / 32) * 32));
    size_t budget = (size_t)smem_optin - 1024;
    const size_t share = (size_t)smem_sm / (size_t)blocks_per_sm;
    if (share < 2048) return plan;
    budget = std::min(budget, share - 2048);
    // the corner indices join the shared memory when they fit (idx_mode 0: never)
    int idx = 1;
    size_t smem = sesm_stream_smem(m, 1);
    if (smem > budget || idx_mode == 0) {
        idx = 0;
        smem = sesm_stream_smem(m, 0);
    }
    if (smem > budget) return plan;
    // the vertices' data joins when it fits (its cached incidences index the fluxes with 16 bits)
    int vc = 0;
    if (m.csr < 65536 && 3 * (size_t)m.slots < 65536 && sesm_stream_smem(m, idx, 1) <= budget) {
        vc = 1;
        smem = sesm_stream_smem(m, idx, 1);
    }
    for (int nonlin = 0; nonlin < 2; nonlin++) {
        void *fn = sesm_stream_kernel(nonlin, idx);
        int occ = 0;
        if (!fn || raise_smem_limit(fn) < (int)smem ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, t, smem) != cudaSuccess || occ < blocks_per_sm) {
            cudaGetLastError();
            return plan;
        }
    }
    plan.slots_per_thread = (m.slots + t - 1) / t;   // rounds of the slot loop (not registers)
    plan.threads = t;
    plan.cached = vc;    // streaming kernels: 1 when the vertices' data is in shared memory
    plan.stream = idx ? 1 : 2;
    plan.blocks_per_sm = blocks_per_sm;
    plan.smem = smem;
    return plan;
}

cudaError_t persistent_prepare_sesm_stream(const PersistentPlan &plan)
{
    for (int nonlin = 0; nonlin < 2; nonlin++) {
        void *fn = sesm_stream_kernel(nonlin, plan.stream == 1);
        if (!fn || raise_smem_limit(fn) < (int)plan.smem) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_persistent_sesm_stream_pack(const DevMesh &m, const DevState &s, const StepArgs &a, int M,
                                               int parity, const PackPlan &pk, int pack_index, cudaStream_t stream)
{
    if (!s.U_x[0] || !s.U_x[1]) return cudaErrorInvalidValue;
    QArgs A;
    A.P = make_pargs(m, s, a, M, parity, pk.mx);
    A.P.pack_base = pk.base;
    A.P.pack_index = pack_index;
    A.U2 = s.U_x[0];
    A.UAB = s.U_x[1];
    A.Shi = s.S_hi;
    A.Slo = s.S_lo;
    A.off_hist = (int)hist_offset(smem_layout(pk.mx));
    A.off_idx = (int)idx_offset(pk.mx);
    A.vmax = pk.mx.vertices;
    A.vcache = pk.plan_sesm.cached;
    if (A.vcache) sesm_stream_smem(pk.mx, pk.plan_sesm.stream == 1, 1, &A.P);
    void *fn = sesm_stream_kernel(a.nonlinear_h, pk.plan_sesm.stream == 1);
    void *args[] = {&A};
    return cudaLaunchCooperativeKernel(fn, dim3(pk.nblocks), dim3(pk.plan_sesm.threads), args, pk.plan_sesm.smem,
                                       stream);
}

}  // namespace sesw
