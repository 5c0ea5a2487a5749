// The persistent step kernel of libsesw with the barotropic viscous regularisation of
// Eq. (viscosity_BT) (sm_103a): one cooperative launch runs the M substeps of Eq. (4.10)
// of a baroclinic step with the forcing R + R_hV(U^m, eta^m) - R_hV(U^0, eta^0), the
// time-mean transport of Eq. (4.12) and the freshwater flux of Eq. (4.5).
#include "sesw_persistent.cuh"

namespace sesw {

namespace {

// ---------------------------------------------------------------------------------
// The viscous flux of a slot needs, across each of its edges, the neighbouring element's
// transport U^m and the elevation eta^m at that element's corner opposite the edge. The
// neighbour can belong to a patch two hops away in the halo graph (its owner waits on a
// patch that waits on this one), and so can that corner. Both are exchanged with the
// tagged words of the SE kernel, in rings of kRing buffers: owner slots publish U^m (two
// words, tag base + 1 + m) and vertices publish eta^m (tag base + m), and a reader takes
// a word only when its tag is the one it needs. A patch runs at most two substeps ahead
// of any patch it reads from, so a writer overwrites a ring entry (tag t by t + kRing)
// only after every reader of tag t has used it. U tags start at base + 1, so a word
// never written (tag 0) is never taken in the first launch. The start value
// R_hV(U^0, eta^0) of each slot stays in registers.
constexpr int kViscThreads = 384;   // registers: 65536 / (2 x 384) = 85 per thread
constexpr int kRing = 4;

struct ViscRefs {
    const int4 *q, *c;          // neighbour owner slots (-1: coast) and h0 bits; opposite corners and h0 bits
    const float4 *a, *b, *r;    // L/d (and h0), L^2/d, frame turns (ROT)
    const float2 *r2;
    unsigned long long *ub;     // kRing x 2 nslot words: U of owner slots
    unsigned long long *xr;     // kRing x nv words: eta of vertices
    long long ub_stride, xr_stride;
    float background, flow;
};

struct VArgs {
    PArgs P;
    ViscRefs V;
};

__device__ __forceinline__ unsigned long long tagged(unsigned tag, float v)
{
    return ((unsigned long long)tag << 32) | __float_as_uint(v);
}

template <int SPT, int NONLIN, int ROT>
__global__ void __launch_bounds__(kViscThreads, 2) k_persistent_visc(VArgs A)
{
    const PArgs &P = A.P;
    const ViscRefs &V = A.V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_abort;
    const int p = P.pack_patch[P.pack_base + blockIdx.x];
    const int T = blockDim.x;
    const int s0 = P.patch_slot[p], ns = P.patch_slot[p + 1] - s0;
    const int nown_s = P.patch_own[p];
    const int v0 = P.patch_v[p], nown = P.patch_v[p + 1] - v0;
    const int hb = P.patch_halo[p], nhalo = P.patch_halo[p + 1] - hb;
    const int c0 = P.vcsr_off[v0], ncsr = P.vcsr_off[v0 + nown] - c0;
    const StepArgs a = P.a;
    const float dt = P.patch_dt[p];
    unsigned *base_word = P.flags + (size_t)(1 + 2 * P.pack_index) * kFlagStride;
    unsigned *exit_count = base_word + kFlagStride;
    const unsigned base = ld_relaxed_gpu(base_word);
    const unsigned abort_val = base + 1u == 0u ? 1u : base + 1u;   // never 0, unique per launch
    const bool publish = p != a.silent_patch;

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
    for (int i = threadIdx.x; i < ns; i += T) {
        // (A_e, H0_e, f dt / 2, 1 / (1 + (f dt / 2)^2))
        const float4 c = P.sc[s0 + i];
        const float aa = c.z * (0.5f * dt);
        s_g[i] = P.sg[s0 + i];
        s_c[i] = make_float4(c.x, c.y, aa, 1.0f / (1.0f + aa * aa));
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
    float2 u[SPT], shi[SPT], slo[SPT], vz[SPT];
#pragma unroll
    for (int j = 0; j < SPT; j++) {
        const int i = threadIdx.x + j * T;
        u[j] = i < ns ? P.U[s0 + i] : make_float2(0.0f, 0.0f);
        shi[j] = make_float2(0.0f, 0.0f);
        slo[j] = make_float2(0.0f, 0.0f);
        vz[j] = make_float2(0.0f, 0.0f);
        // U^0 of owner slots for the neighbours' viscous fluxes
        if (i < nown_s && publish) {
            unsigned long long *w = V.ub + 2 * (size_t)(s0 + i);
            st_relaxed_gpu_u64(w, tagged(base + 1u, u[j].x));
            st_relaxed_gpu_u64(w + 1, tagged(base + 1u, u[j].y));
        }
    }
    __syncthreads();

    const float one_p_theta = 1.0f + a.theta;
    bool ok = true;
    for (int m = 0; m < P.M; m++) {
        const unsigned teta = base + (unsigned)m, tu = base + 1u + (unsigned)m;
        const unsigned long long *xs = V.xr + (size_t)(m % kRing) * V.xr_stride;
        const unsigned long long *us = V.ub + (size_t)(m % kRing) * V.ub_stride;
        unsigned long long *uout = V.ub + (size_t)((m + 1) % kRing) * V.ub_stride;
        const bool more = m + 1 < P.M;
#pragma unroll
        for (int j = 0; j < SPT; j++) {
            const int i = threadIdx.x + j * T;
            if (i >= ns) continue;
            const int s = s0 + i;
            const float4 g = s_g[i], c = s_c[i];
            const float2 r = s_r[i];
            const ushort4 l = s_l[i];
            const int4 tq = V.q[s], tc = V.c[s];
            const float4 ta = V.a[s], tb = V.b[s];
            // every exchanged value of the slot is requested before any is waited for
            const int hc[3] = {l.x < nown ? -1 : s_halo[l.x - nown], l.y < nown ? -1 : s_halo[l.y - nown],
                               l.z < nown ? -1 : s_halo[l.z - nown]};
            const int nq[3] = {tq.x, tq.y, tq.z};
            const int oc[3] = {tc.x, tc.y, tc.z};
            unsigned long long wc[3], wu[3][2], wo[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                wc[k] = (m > 0 && hc[k] >= 0) ? ld_relaxed_gpu_u64(xs + hc[k]) : 0ull;
                if (nq[k] >= 0) {
                    wu[k][0] = ld_relaxed_gpu_u64(us + 2 * (size_t)nq[k]);
                    wu[k][1] = ld_relaxed_gpu_u64(us + 2 * (size_t)nq[k] + 1);
                } else {
                    wu[k][0] = wu[k][1] = 0ull;
                }
                const bool own_oc = oc[k] >= v0 && oc[k] < v0 + nown;
                wo[k] = (NONLIN && m > 0 && nq[k] >= 0 && !own_oc) ? ld_relaxed_gpu_u64(xs + oc[k]) : 0ull;
            }
            const unsigned short lc[3] = {l.x, l.y, l.z};
            float e[3];
#pragma unroll
            for (int k = 0; k < 3; k++)
                e[k] = (m == 0 || hc[k] < 0) ? seta[lc[k]] : halo_eta(P, xs, hc[k], wc[k], teta, abort_val, ok);
            const float d0 = e[0] - e[2], d1 = e[1] - e[2];
            const float gx = d0 * g.x + d1 * g.z;
            const float gy = d0 * g.y + d1 * g.w;
            float H = c.y;
            if (NONLIN) H += (e[0] + e[1] + e[2]) * (1.0f / 3.0f);
            // R_hV(U^m, eta^m) of the slot: two-point fluxes across its edges
            const float ux = u[j].x / H, uy = u[j].y / H;
            const float h0[3] = {__int_as_float(tq.w), __int_as_float(tc.w), ta.w};
            const float la[3] = {ta.x, ta.y, ta.z};
            const float lb[3] = {tb.x, tb.y, tb.z};
            float cs[3] = {1.0f, 1.0f, 1.0f}, sn[3] = {0.0f, 0.0f, 0.0f};
            if (ROT) {
                const float4 rr = V.r[s];
                const float2 r2 = V.r2[s];
                cs[0] = rr.x;
                sn[0] = rr.y;
                cs[1] = rr.z;
                sn[1] = rr.w;
                cs[2] = r2.x;
                sn[2] = r2.y;
            }
            float fvx = 0.0f, fvy = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (nq[k] < 0) continue;
                float Hn = h0[k];
                if (NONLIN) {
                    float eo;
                    if (oc[k] >= v0 && oc[k] < v0 + nown)
                        eo = seta[oc[k] - v0];
                    else if (m == 0)
                        eo = __ldg(P.eta_in + oc[k]);
                    else
                        eo = halo_eta(P, xs, oc[k], wo[k], teta, abort_val, ok);
                    Hn += (e[k] + e[(k + 1) % 3] + eo) * (1.0f / 3.0f);
                }
                const float qx = halo_eta(P, us, 2 * nq[k], wu[k][0], tu, abort_val, ok);
                const float qy = halo_eta(P, us, 2 * nq[k] + 1, wu[k][1], tu, abort_val, ok);
                const float nx = qx / Hn, ny = qy / Hn;
                float dx, dy;
                if (ROT) {
                    dx = (cs[k] * nx - sn[k] * ny) - ux;
                    dy = (sn[k] * nx + cs[k] * ny) - uy;
                } else {
                    dx = nx - ux;
                    dy = ny - uy;
                }
                const float kq = 0.5f * (H + Hn) * (V.background * la[k] + V.flow * sqrtf(dx * dx + dy * dy) * lb[k]);
                fvx += kq * dx;
                fvy += kq * dy;
            }
            const float2 Vv = make_float2(fvx / c.x, fvy / c.x);
            float2 rr = r;
            if (m == 0)
                vz[j] = Vv;   // R' = R + (V - V) = R
            else
                rr = make_float2(r.x + (Vv.x - vz[j].x), r.y + (Vv.y - vz[j].y));
            // Eq. (4.10), first row, with Crank-Nicolson Coriolis, and the theta-weighted flux
            const float gH = a.g * H;
            const float aa = c.z;
            const float rx = u[j].x + aa * u[j].y + dt * (rr.x - gH * gx);
            const float ry = u[j].y - aa * u[j].x + dt * (rr.y - gH * gy);
            const float nx = (rx + aa * ry) * c.w;
            const float ny = (ry - aa * rx) * c.w;
            const float fx = one_p_theta * nx - a.theta * u[j].x;
            const float fy = one_p_theta * ny - a.theta * u[j].y;
            u[j] = make_float2(nx, ny);
            if (i < nown_s) {
                two_sum_acc(shi[j].x, slo[j].x, fx);
                two_sum_acc(shi[j].y, slo[j].y, fy);
                if (more && publish) {
                    unsigned long long *w = uout + 2 * (size_t)s;
                    st_relaxed_gpu_u64(w, tagged(tu + 1u, nx));
                    st_relaxed_gpu_u64(w + 1, tagged(tu + 1u, ny));
                }
            }
            const float wgt = dt * c.x;
            const float q0 = wgt * (fx * g.x + fy * g.y);
            const float q1 = wgt * (fx * g.z + fy * g.w);
            sflux[3 * i + 0] = q0;
            sflux[3 * i + 1] = q1;
            sflux[3 * i + 2] = -(q0 + q1);
        }
        if (!ok) s_abort = 1;
        __syncthreads();
        if (s_abort) break;

        // vertex pass; the new elevation of own vertices also goes to the ring
        unsigned long long *xout = V.xr + (size_t)((m + 1) % kRing) * V.xr_stride;
        bool bad = false;
        for (int i = threadIdx.x; i < nown; i += T) {
            float sum = 0.0f;
            const int k1 = s_off[i + 1];
            for (int k = s_off[i]; k < k1; k++) sum += sflux[s_csr[k]];
            float e = seta[i] + sum * s_inv[i];
            if (P.W) e -= dt * __ldg(P.W + v0 + i);
            if (P.eta_sum) P.eta_sum[v0 + i] += seta[i];
            seta[i] = e;
            if (more && publish) st_relaxed_gpu_u64(xout + v0 + i, tagged(teta + 1u, e));
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

template <int NONLIN, int ROT>
void *visc_fn(int spt)
{
    switch (spt) {
    case 1: return (void *)k_persistent_visc<1, NONLIN, ROT>;
    case 2: return (void *)k_persistent_visc<2, NONLIN, ROT>;
    case 3: return (void *)k_persistent_visc<3, NONLIN, ROT>;
    case 4: return (void *)k_persistent_visc<4, NONLIN, ROT>;
    default: return nullptr;
    }
}

void *visc_kernel(int spt, int nonlin, int rot)
{
    if (rot) return nonlin ? visc_fn<1, 1>(spt) : visc_fn<0, 1>(spt);
    return nonlin ? visc_fn<1, 0>(spt) : visc_fn<0, 0>(spt);
}

}  // namespace

PersistentPlan persistent_plan_visc(const PatchMax &m, int blocks_per_sm)
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
    // fewest slots per thread such that one block of at most kViscThreads covers the
    // largest patch
    int spt = 0, t = 0;
    for (int cand = 1; cand <= 4; cand++) {
        const int need = (m.slots + cand - 1) / cand;
        const int tt = std::max(32, ((need + 31) / 32) * 32);
        if (tt <= kViscThreads) {
            spt = cand;
            t = tt;
            break;
        }
    }
    if (!spt) return plan;
    const SmemLayout L = smem_layout(m);
    size_t budget = (size_t)smem_optin - 1024;
    const size_t share = (size_t)smem_sm / (size_t)blocks_per_sm;
    if (share < 2048) return plan;
    budget = std::min(budget, share - 2048);
    if (L.total_cached > budget || m.csr >= 65536 || m.slots >= 16384) return plan;
    for (int nonlin = 0; nonlin < 2; nonlin++)
        for (int rot = 0; rot < 2; rot++) {
            void *fn = visc_kernel(spt, nonlin, rot);
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

cudaError_t persistent_prepare_visc(const PersistentPlan &plan)
{
    for (int nonlin = 0; nonlin < 2; nonlin++)
        for (int rot = 0; rot < 2; rot++) {
            void *fn = visc_kernel(plan.slots_per_thread, nonlin, rot);
            if (!fn || raise_smem_limit(fn) < (int)plan.smem) return cudaErrorInvalidValue;
        }
    return cudaSuccess;
}

size_t persistent_visc_ring_words(int nv, int nslot) { return (size_t)kRing * ((size_t)nv + 2 * (size_t)nslot); }

cudaError_t launch_persistent_visc(const DevMesh &m, const DevState &s, const StepArgs &a, const ViscArgs &va,
                                   unsigned long long *ring, int M, int parity, const std::vector<PackPlan> &packs,
                                   cudaStream_t stream)
{
    VArgs A;
    A.V.q = m.visc_q;
    A.V.c = m.visc_c;
    A.V.a = m.visc_a;
    A.V.b = m.visc_b;
    A.V.r = m.visc_r;
    A.V.r2 = m.visc_r2;
    A.V.xr = ring;
    A.V.xr_stride = m.nv;
    A.V.ub = ring + (size_t)kRing * m.nv;
    A.V.ub_stride = 2 * (long long)m.nslot;
    A.V.background = va.background;
    A.V.flow = va.flow;
    for (size_t k = 0; k < packs.size(); k++) {
        const PackPlan &pk = packs[k];
        const PersistentPlan &plan = pk.plan_visc;
        void *fn = visc_kernel(plan.slots_per_thread, a.nonlinear_h, m.visc_rot);
        if (!fn) return cudaErrorInvalidValue;
        A.P = make_pargs(m, s, a, M, parity, pk.mx);
        A.P.pack_base = pk.base;
        A.P.pack_index = (int)k;
        void *args[] = {&A};
        cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(pk.nblocks), dim3(plan.threads), args, plan.smem, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sesw
