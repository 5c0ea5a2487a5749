// The SESM step kernel of libsesw (sm_103a): one cooperative launch runs a baroclinic
// step of the AB3-AM4 substep of Eqs. (4.7)-(4.8), with the time-mean transport of Eq.
// (4.12) and the freshwater flux of Eq. (4.5).
#include "sesw_persistent.cuh"

namespace sesw {

namespace {

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
// same tagged words as the SE kernel (tag base + m for substep m, m = 1 .. M). As in the SE
// kernel, the halo words of a thread's last-round slot are requested after its first round.
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
    const StepArgs a = P.a;
    const float dt = P.patch_dt[p];
    unsigned *base_word = P.flags + (size_t)(1 + 2 * P.pack_index) * kFlagStride;
    unsigned *exit_count = base_word + kFlagStride;
    const unsigned base = ld_relaxed_gpu(base_word);
    const unsigned abort_val = base + 1u == 0u ? 1u : base + 1u;   // never 0, unique per launch

    float *sem = reinterpret_cast<float *>(smem_raw);   // eta_AM of the own vertices, then of the halo
    float *sflux = reinterpret_cast<float *>(smem_raw + P.off_flux);
    float4 *s_g = reinterpret_cast<float4 *>(smem_raw + P.off_g);
    float4 *s_c = reinterpret_cast<float4 *>(smem_raw + P.off_c);
    float2 *s_r = reinterpret_cast<float2 *>(smem_raw + P.off_r);
    ushort4 *s_l = reinterpret_cast<ushort4 *>(smem_raw + P.off_l);
    float *s_inv = reinterpret_cast<float *>(smem_raw + P.off_inv);
    int *s_halo = reinterpret_cast<int *>(smem_raw + P.off_halo);

    for (int i = threadIdx.x; i < ns; i += T) {
        s_g[i] = P.sg[s0 + i];
        s_c[i] = P.sc[s0 + i];
        s_r[i] = P.R[s0 + i];
        s_l[i] = P.sl[s0 + i];
    }
    cache_incidences(P, smem_raw, v0, nown);
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
        const float2 F = sesm_ab3(u0, ua, ub, a.ab0, a.ab1, a.ab2);
        if (i < nown_s) {
            two_sum_acc2(shi[j], slo[j], F);
        }
        corner_fluxes(F, g, __fmul_rn(dt, area), sflux + 3 * i);
        uab[j] = F;
    };
    bool ok = true;
    // momentum update of slot i (round j) from its corner eta_AM
    auto slot = [&](int j, int i, float e0, float e1, float e2, bool vertex) {
        const float4 g = s_g[i], c = s_c[i];
        const float2 r = s_r[i];
        const float2 u0 = sesm_momentum<NONLIN>(e0, e1, e2, g, c.y, a.g, c.z, dt, r, u1[j], uab[j]);
        if (vertex) transport(j, i, u0, u1[j], u2[j], g, c.x);
        u2[j] = u1[j];
        u1[j] = u0;
    };
    auto halo_of = [&](unsigned l) { return (int)l < nown ? -1 : s_halo[l - nown]; };

    const int npre = nint >= T ? (nint / T) * T : nint;
    // the last round's slot, when it is not a whole-round interior one: its halo words are
    // requested right after the first round
    const int ilast = threadIdx.x + (SPT - 1) * T;
    const bool early = SPT > 1 && ilast >= npre && ilast < ns;
    // one thread per halo vertex requests its tagged word before the interior rounds and stores
    // the value after the eta_AM of the own vertices; the other slots then read every corner
    // from shared memory (patches with more halo vertices than threads keep the reads per slot)
    const bool hpre = nhalo <= T;
    for (int m = 0; m <= P.M; m++) {
        const bool vertex = m < P.M;
        if (m == 0) {
            // no momentum update: U_AB^0 from level 0 and its aliases
#pragma unroll
            for (int j = 0; j < SPT; j++) {
                const int i = threadIdx.x + j * T;
                if (i < ns) transport(j, i, u1[j], u1[j], u1[j], s_g[i], s_c[i].x);
            }
        } else if (hpre) {
            const unsigned long long *xs = P.xb[m & 1];
            const int hv = (int)threadIdx.x < nhalo ? s_halo[threadIdx.x] : -1;
            const unsigned long long hw = hv >= 0 ? ld_relaxed_gpu_u64(xs + hv) : 0ull;
#pragma unroll
            for (int j = 0; j < SPT; j++) {
                const int i = threadIdx.x + j * T;
                if (i < npre) {
                    const ushort4 l = s_l[i];
                    slot(j, i, sem[l.x], sem[l.y], sem[l.z], vertex);
                }
            }
            if (hv >= 0) sem[nown + threadIdx.x] = halo_eta(P, xs, hv, hw, base + (unsigned)m, abort_val, ok);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < SPT; j++) {
                const int i = threadIdx.x + j * T;
                if (i >= npre && i < ns) {
                    const ushort4 l = s_l[i];
                    slot(j, i, sem[l.x], sem[l.y], sem[l.z], vertex);
                }
            }
            if (!ok) s_abort = 1;
        } else {
            const unsigned tag = base + (unsigned)m;
            const unsigned long long *xs = P.xb[m & 1];
            unsigned long long q0 = 0ull, q1 = 0ull, q2 = 0ull;
#pragma unroll
            for (int j = 0; j < SPT; j++) {
                const int i = threadIdx.x + j * T;
                if (SPT > 1 && j == SPT - 1) {
                    if (early) {
                        const ushort4 l = s_l[i];
                        const int h0 = halo_of(l.x), h1 = halo_of(l.y), h2 = halo_of(l.z);
                        const float e0 = h0 < 0 ? sem[l.x] : halo_eta(P, xs, h0, q0, tag, abort_val, ok);
                        const float e1 = h1 < 0 ? sem[l.y] : halo_eta(P, xs, h1, q1, tag, abort_val, ok);
                        const float e2 = h2 < 0 ? sem[l.z] : halo_eta(P, xs, h2, q2, tag, abort_val, ok);
                        slot(j, i, e0, e1, e2, vertex);
                    } else if (i < npre) {
                        const ushort4 l = s_l[i];
                        slot(j, i, sem[l.x], sem[l.y], sem[l.z], vertex);
                    }
                } else if (i < ns) {
                    const ushort4 l = s_l[i];
                    if (i < npre) {
                        slot(j, i, sem[l.x], sem[l.y], sem[l.z], vertex);
                    } else {
                        const int h0 = halo_of(l.x), h1 = halo_of(l.y), h2 = halo_of(l.z);
                        const unsigned long long w0 = h0 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h0);
                        const unsigned long long w1 = h1 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h1);
                        const unsigned long long w2 = h2 < 0 ? 0ull : ld_relaxed_gpu_u64(xs + h2);
                        const float e0 = h0 < 0 ? sem[l.x] : halo_eta(P, xs, h0, w0, tag, abort_val, ok);
                        const float e1 = h1 < 0 ? sem[l.y] : halo_eta(P, xs, h1, w1, tag, abort_val, ok);
                        const float e2 = h2 < 0 ? sem[l.z] : halo_eta(P, xs, h2, w2, tag, abort_val, ok);
                        slot(j, i, e0, e1, e2, vertex);
                    }
                }
                if (j == 0 && early) {
                    const ushort4 l = s_l[ilast];
                    const int h0 = halo_of(l.x), h1 = halo_of(l.y), h2 = halo_of(l.z);
                    if (h0 >= 0) q0 = ld_relaxed_gpu_u64(xs + h0);
                    if (h1 >= 0) q1 = ld_relaxed_gpu_u64(xs + h1);
                    if (h2 >= 0) q2 = ld_relaxed_gpu_u64(xs + h2);
                }
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
#pragma unroll
        for (int k = 0; k < kSesmVpt; k++) {
            const int i = threadIdx.x + k * T;
            if (i < nown) {
                const float sum = cached_flux_sum(P, smem_raw, i);
                float e = vertex_eta(eh0[k], sum, s_inv[i]);
                if (P.W) e = __fmaf_rn(-dt, __ldg(P.W + v0 + i), e);
                const float em = sesm_am4(e, eh0[k], eh1[k], eh2[k], a.am0, a.am1, a.am2, a.am3);
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

}  // namespace

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
    // one cooperative launch per pack, each with its own plan, layout and tag base
    for (size_t k = 0; k < packs.size(); k++) {
        const PackPlan &pk = packs[k];
        if (pk.plan_sesm.stream) {
            const cudaError_t e = launch_persistent_sesm_stream_pack(m, s, a, M, parity, pk, (int)k, stream);
            if (e != cudaSuccess) return e;
            continue;
        }
        void *fn = sesm_kernel(pk.plan_sesm.slots_per_thread, a.nonlinear_h);
        if (!fn) return cudaErrorInvalidValue;
        PArgs P = make_pargs(m, s, a, M, parity, pk.mx);
        P.pack_base = pk.base;
        P.pack_index = (int)k;
        void *args[] = {&P};
        cudaError_t e =
            cudaLaunchCooperativeKernel(fn, dim3(pk.nblocks), dim3(pk.plan_sesm.threads), args, pk.plan_sesm.smem, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sesw
