// Host-side mesh preparation for libsesw: validation, P1 geometry, Hilbert
// ordering, vertex patches with guest element copies, per-vertex incidence lists.
//
// Geometry (the paper defers the spatial discretisation to FESOM2's finite-volume
// layout: scalars on vertices with median-dual control volumes, transports on
// triangles): for a counter-clockwise triangle (a, b, c) with area A_e, the
// gradient of the linear basis function of corner a is rot90(p_c - p_b) / (2 A_e),
// rot90(x, y) = (-y, x). The median-dual area of a vertex is the sum of A_e/3 over
// its triangles.
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "sesw_internal.h"

namespace sesw {

// Hilbert index of (x, y) on a 2^bits x 2^bits grid. At each level the quadrant
// digit is read from the current bit of x and y, then the lower bits are rotated
// or reflected so the sub-square is traversed in the curve's orientation.
uint64_t hilbert2d(uint32_t x, uint32_t y, int bits)
{
    uint64_t d = 0;
    for (int b = bits - 1; b >= 0; b--) {
        uint32_t s = 1u << b;
        uint32_t rx = (x & s) ? 1u : 0u;
        uint32_t ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * (uint64_t)s * (uint64_t)((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = ~x;
                y = ~y;
            }
            uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// Hilbert index in 3-D, following Skilling's transpose formulation (J. Skilling,
// "Programming the Hilbert curve", AIP Conf. Proc. 707, 2004): undo the excess
// rotations level by level, Gray-encode, then interleave the bits of the three
// transposed coordinates from the most significant level down.
uint64_t hilbert3d(uint32_t x, uint32_t y, uint32_t z, int bits)
{
    uint32_t X[3] = {x, y, z};
    const int n = 3;
    uint32_t top = 1u << (bits - 1);
    for (uint32_t q = top; q > 1; q >>= 1) {
        uint32_t p = q - 1;
        for (int i = 0; i < n; i++) {
            if (X[i] & q) {
                X[0] ^= p;
            } else {
                uint32_t t = (X[0] ^ X[i]) & p;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    for (int i = 1; i < n; i++) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
        if (X[n - 1] & q) t ^= q - 1;
    for (int i = 0; i < n; i++) X[i] ^= t;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; b--)
        for (int i = 0; i < n; i++) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

static bool finite(double v) { return std::isfinite(v); }

static void fmt(std::string &err, const char *f, long long a, double b = 0.0)
{
    char buf[256];
    snprintf(buf, sizeof buf, f, a, b);
    err = buf;
}

int prepare_mesh(const sesw_mesh &m, int patch_vertices, HostMesh &out, std::string &err)
{
    const int nv = m.nv, ne = m.ne;
    if (nv < 1 || ne < 1) { err = "mesh needs nv >= 1 and ne >= 1"; return SESW_EINVAL; }
    if (!m.tri || !m.xy || !m.depth || !m.coriolis) { err = "mesh has a NULL array"; return SESW_EINVAL; }
    if ((long long)ne * 3 >= (1ll << 31) || (long long)nv >= (1ll << 30)) {
        err = "mesh too large for 32-bit indexing";
        return SESW_EINVAL;
    }
    if (patch_vertices < 32) patch_vertices = 32;

    // ---- element checks and FP64 geometry (caller order)
    std::vector<double> A(ne), gph(6 * (size_t)ne);
    for (int e = 0; e < ne; e++) {
        const int32_t *t = m.tri + 3 * (size_t)e;
        for (int k = 0; k < 3; k++)
            if (t[k] < 0 || t[k] >= nv) { fmt(err, "triangle %lld has a vertex index out of range", e); return SESW_EINVAL; }
        if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2]) { fmt(err, "triangle %lld repeats a vertex", e); return SESW_EINVAL; }
        const double *p = m.xy + 6 * (size_t)e;
        for (int k = 0; k < 6; k++)
            if (!finite(p[k])) { fmt(err, "triangle %lld has a non-finite coordinate", e); return SESW_EINVAL; }
        double twoA = (p[2] - p[0]) * (p[5] - p[1]) - (p[4] - p[0]) * (p[3] - p[1]);
        if (!(twoA > 0.0)) { fmt(err, "triangle %lld is not counter-clockwise with positive area", e); return SESW_EINVAL; }
        A[e] = 0.5 * twoA;
        for (int k = 0; k < 3; k++) {
            const double *pb = p + 2 * ((k + 1) % 3), *pc = p + 2 * ((k + 2) % 3);
            gph[6 * (size_t)e + 2 * k] = -(pc[1] - pb[1]) / twoA;
            gph[6 * (size_t)e + 2 * k + 1] = (pc[0] - pb[0]) / twoA;
        }
        if (!finite(m.coriolis[e])) { fmt(err, "triangle %lld has a non-finite Coriolis parameter", e); return SESW_EINVAL; }
    }
    for (int v = 0; v < nv; v++)
        if (!(m.depth[v] > 0.0) || !finite(m.depth[v])) { fmt(err, "vertex %lld has a depth that is not positive and finite", v); return SESW_EINVAL; }

    // ---- edges: each shared by at most two triangles, in opposite directions. The
    // off-diagonal stiffness of each edge, K_ab = sum_e A_e H0_e dphi_a . dphi_b, is
    // summed on the way for the Gershgorin bound below.
    std::vector<double> kdiag(nv, 0.0), koff(nv, 0.0);
    std::vector<int> nb_c(3 * (size_t)ne, -1);    // neighbour across edge (corner k, corner k+1), caller ids
    {
        struct HE { uint64_t key; double k; int ek; };
        std::vector<HE> he(3 * (size_t)ne);
        for (int e = 0; e < ne; e++) {
            const int32_t *t = m.tri + 3 * (size_t)e;
            const double *g = gph.data() + 6 * (size_t)e;
            const double h0 = (m.depth[t[0]] + m.depth[t[1]] + m.depth[t[2]]) / 3.0;
            for (int k = 0; k < 3; k++) {
                int kn = (k + 1) % 3;
                uint32_t a = (uint32_t)t[k], b = (uint32_t)t[kn];
                uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
                // low bit: direction (1 when traversed from the higher to the lower index)
                he[3 * (size_t)e + k].key = (((uint64_t)lo * (uint64_t)nv + hi) << 1) | (a > b ? 1u : 0u);
                he[3 * (size_t)e + k].k = A[e] * h0 * (g[2 * k] * g[2 * kn] + g[2 * k + 1] * g[2 * kn + 1]);
                he[3 * (size_t)e + k].ek = 3 * e + k;
                kdiag[t[k]] += A[e] * h0 * (g[2 * k] * g[2 * k] + g[2 * k + 1] * g[2 * k + 1]);
            }
        }
        std::sort(he.begin(), he.end(), [](const HE &x, const HE &y) { return x.key < y.key; });
        for (size_t i = 0; i < he.size();) {
            size_t j = i;
            while (j < he.size() && (he[j].key >> 1) == (he[i].key >> 1)) j++;
            if (j - i > 2) { err = "an edge is shared by more than two triangles"; return SESW_EINVAL; }
            if (j - i == 2 && (he[i].key & 1u) == (he[i + 1].key & 1u)) {
                err = "two triangles traverse a shared edge in the same direction (inconsistent orientation)";
                return SESW_EINVAL;
            }
            if (j - i == 2) {
                nb_c[he[i].ek] = he[i + 1].ek / 3;
                nb_c[he[i + 1].ek] = he[i].ek / 3;
            }
            double kab = 0.0;
            for (size_t q = i; q < j; q++) kab += he[q].k;
            uint64_t pair = he[i].key >> 1;
            koff[pair / (uint64_t)nv] += fabs(kab);
            koff[pair % (uint64_t)nv] += fabs(kab);
            i = j;
        }
        // the caller's edge table, when given, must list exactly these edges with their triangles
        if (m.edge_v || m.edge_e || m.ned != 0) {
            if (!m.edge_v || !m.edge_e) { err = "edge_v and edge_e must be given together"; return SESW_EINVAL; }
            std::vector<uint64_t> keys;
            std::vector<std::pair<int, int>> sides;
            for (size_t i = 0; i < he.size();) {
                size_t j = i + 1;
                while (j < he.size() && (he[j].key >> 1) == (he[i].key >> 1)) j++;
                const int a = he[i].ek / 3, b = j - i == 2 ? he[i + 1].ek / 3 : -1;
                keys.push_back(he[i].key >> 1);
                sides.push_back({std::min(a, b), std::max(a, b)});
                i = j;
            }
            if ((size_t)m.ned != keys.size()) {
                fmt(err, "the edge table lists %lld edges; the triangles have %.0f", m.ned, (double)keys.size());
                return SESW_EINVAL;
            }
            std::vector<char> seen(keys.size(), 0);
            for (int k = 0; k < m.ned; k++) {
                const int a = m.edge_v[2 * (size_t)k], b = m.edge_v[2 * (size_t)k + 1];
                if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) { fmt(err, "edge %lld has a bad vertex", k); return SESW_EINVAL; }
                const uint64_t key = (uint64_t)std::min(a, b) * (uint64_t)nv + (uint64_t)std::max(a, b);
                const size_t q = std::lower_bound(keys.begin(), keys.end(), key) - keys.begin();
                if (q == keys.size() || keys[q] != key) { fmt(err, "edge %lld is not a side of any triangle", k); return SESW_EINVAL; }
                if (seen[q]) { fmt(err, "edge %lld is listed twice", k); return SESW_EINVAL; }
                seen[q] = 1;
                const int ea = m.edge_e[2 * (size_t)k], eb = m.edge_e[2 * (size_t)k + 1];
                if (std::make_pair(std::min(ea, eb), std::max(ea, eb)) != sides[q]) {
                    fmt(err, "edge %lld does not list the triangles on its two sides", k);
                    return SESW_EINVAL;
                }
            }
        }
    }

    // ---- median-dual areas; every vertex must be a corner of some triangle
    std::vector<double> Av(nv, 0.0);
    for (int e = 0; e < ne; e++)
        for (int k = 0; k < 3; k++) Av[m.tri[3 * (size_t)e + k]] += A[e] / 3.0;
    for (int v = 0; v < nv; v++)
        if (!(Av[v] > 0.0)) { fmt(err, "vertex %lld is not a corner of any triangle", v); return SESW_EINVAL; }
    // the caller's areas, when given, must be the derived ones
    auto area_ok = [](double given, double want) { return fabs(given - want) <= 1e-12 * want; };
    if (m.area_e)
        for (int e = 0; e < ne; e++)
            if (!area_ok(m.area_e[e], A[e])) {
                fmt(err, "area_e[%lld] differs from the area of the triangle's corners (%.17g)", e, A[e]);
                return SESW_EINVAL;
            }
    if (m.area_v)
        for (int v = 0; v < nv; v++)
            if (!area_ok(m.area_v[v], Av[v])) {
                fmt(err, "area_v[%lld] differs from the median-dual area (%.17g)", v, Av[v]);
                return SESW_EINVAL;
            }

    // ---- vertex order along a Hilbert curve
    std::vector<int> vperm(nv);
    std::iota(vperm.begin(), vperm.end(), 0);
    if (m.pos) {
        bool flat = true;
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int v = 0; v < nv; v++)
            for (int c = 0; c < 3; c++) {
                double x = m.pos[3 * (size_t)v + c];
                if (!finite(x)) { fmt(err, "vertex %lld has a non-finite position", v); return SESW_EINVAL; }
                lo[c] = std::min(lo[c], x);
                hi[c] = std::max(hi[c], x);
            }
        if (hi[2] - lo[2] > 0.0) flat = false;
        double span = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
        if (span <= 0.0) span = 1.0;
        const int bits = 16;
        const double scale = ((1u << bits) - 1) / span;
        std::vector<uint64_t> key(nv);
        for (int v = 0; v < nv; v++) {
            uint32_t q[3];
            for (int c = 0; c < 3; c++) q[c] = (uint32_t)((m.pos[3 * (size_t)v + c] - lo[c]) * scale);
            key[v] = flat ? hilbert2d(q[0], q[1], bits) : hilbert3d(q[0], q[1], q[2], bits);
        }
        std::stable_sort(vperm.begin(), vperm.end(), [&](int a, int b) { return key[a] < key[b]; });
    }
    std::vector<int> vinv(nv);
    for (int i = 0; i < nv; i++) vinv[vperm[i]] = i;

    // ---- patches: balanced contiguous ranges of the ordered vertices
    int npatch = (nv + patch_vertices - 1) / patch_vertices;
    std::vector<int> patch_v(npatch + 1);
    for (int p = 0; p <= npatch; p++) patch_v[p] = (int)((long long)p * nv / npatch);
    std::vector<int> vpatch(nv);
    int maxpv = 0;
    for (int p = 0; p < npatch; p++) {
        for (int v = patch_v[p]; v < patch_v[p + 1]; v++) vpatch[v] = p;
        maxpv = std::max(maxpv, patch_v[p + 1] - patch_v[p]);
    }
    // Inside each patch, the vertices that another patch reads (corners of elements that
    // also touch another patch) come first, keeping the curve order otherwise: the
    // persistent kernel's vertex pass then publishes all of them in its first round.
    {
        std::vector<char> exported(nv, 0);
        for (int e = 0; e < ne; e++) {
            const int c[3] = {vinv[m.tri[3 * (size_t)e]], vinv[m.tri[3 * (size_t)e + 1]],
                              vinv[m.tri[3 * (size_t)e + 2]]};
            for (int k = 0; k < 3; k++)
                for (int j = 0; j < 3; j++)
                    if (vpatch[c[k]] != vpatch[c[j]]) exported[c[k]] = 1;
        }
        std::vector<int> order(nv);
        for (int p = 0; p < npatch; p++) {
            int w = patch_v[p];
            for (int pass = 0; pass < 2; pass++)
                for (int v = patch_v[p]; v < patch_v[p + 1]; v++)
                    if ((exported[v] != 0) == (pass == 0)) order[w++] = vperm[v];
        }
        vperm.swap(order);
        for (int i = 0; i < nv; i++) vinv[vperm[i]] = i;
    }

    // ---- element order: by owner patch (patch of the lowest new corner), then corners
    struct EK { int lo, mid, hi, e; };
    std::vector<EK> ek(ne);
    for (int e = 0; e < ne; e++) {
        int c[3] = {vinv[m.tri[3 * (size_t)e]], vinv[m.tri[3 * (size_t)e + 1]], vinv[m.tri[3 * (size_t)e + 2]]};
        std::sort(c, c + 3);
        ek[e] = {c[0], c[1], c[2], e};
    }
    std::sort(ek.begin(), ek.end(), [](const EK &a, const EK &b) {
        if (a.lo != b.lo) return a.lo < b.lo;
        if (a.mid != b.mid) return a.mid < b.mid;
        if (a.hi != b.hi) return a.hi < b.hi;
        return a.e < b.e;
    });
    std::vector<int> eperm(ne), einv(ne);
    for (int i = 0; i < ne; i++) { eperm[i] = ek[i].e; einv[ek[i].e] = i; }
    std::vector<int> owner(ne);
    for (int i = 0; i < ne; i++) owner[i] = vpatch[ek[i].lo];

    // ---- guests: (patch, element) pairs for patches that touch but do not own an element
    std::vector<std::pair<int, int>> guests;
    guests.reserve((size_t)ne / 4);
    for (int i = 0; i < ne; i++) {
        int ps[3] = {vpatch[ek[i].lo], vpatch[ek[i].mid], vpatch[ek[i].hi]};
        for (int k = 0; k < 3; k++) {
            int q = ps[k];
            if (q == owner[i]) continue;
            bool dup = false;
            for (int j = 0; j < k; j++) dup |= (ps[j] == q);
            if (!dup) guests.push_back({q, i});
        }
    }
    std::sort(guests.begin(), guests.end());

    // ---- slots
    std::vector<int> own_begin(npatch + 1, 0);
    for (int i = 0; i < ne; i++) own_begin[owner[i] + 1]++;
    for (int p = 0; p < npatch; p++) own_begin[p + 1] += own_begin[p];
    std::vector<int> g_begin(npatch + 1, 0);
    for (auto &g : guests) g_begin[g.first + 1]++;
    for (int p = 0; p < npatch; p++) g_begin[p + 1] += g_begin[p];

    const int nslot = ne + (int)guests.size();
    std::vector<int> patch_slot(npatch + 1), patch_own(npatch);
    patch_slot[0] = 0;
    int maxslots = 0;
    for (int p = 0; p < npatch; p++) {
        patch_own[p] = own_begin[p + 1] - own_begin[p];
        int n = patch_own[p] + (g_begin[p + 1] - g_begin[p]);
        patch_slot[p + 1] = patch_slot[p] + n;
        maxslots = std::max(maxslots, n);
    }
    if (maxslots >= (1 << 28)) { err = "a patch has too many element slots"; return SESW_EINVAL; }

    // Slot order inside a patch: owned elements whose corners are all the patch's own
    // vertices ("interior"), then the other owned elements, then guests. Interior slots
    // need no halo elevation, so the persistent kernel updates them while it waits for
    // its neighbours.
    std::vector<int> slot_elem(nslot);
    std::vector<char> slot_guest(nslot, 0);
    std::vector<int> patch_int(npatch, 0);
    for (int p = 0; p < npatch; p++) {
        int s = patch_slot[p];
        for (int pass = 0; pass < 2; pass++)
            for (int i = own_begin[p]; i < own_begin[p + 1]; i++) {
                const bool interior = vpatch[ek[i].lo] == p && vpatch[ek[i].mid] == p && vpatch[ek[i].hi] == p;
                if (interior == (pass == 0)) {
                    slot_elem[s++] = i;
                    if (interior) patch_int[p]++;
                }
            }
        for (int k = g_begin[p]; k < g_begin[p + 1]; k++) { slot_guest[s] = 1; slot_elem[s++] = guests[k].second; }
    }

    out = HostMesh();
    out.nv = nv;
    out.ne = ne;
    out.npatch = npatch;
    out.nslot = nslot;
    out.max_patch_slots = maxslots;
    out.max_patch_vertices = maxpv;
    out.patch_vertices = patch_vertices;
    out.vperm = vperm;
    out.eperm = eperm;
    out.patch_v = patch_v;
    out.patch_slot = patch_slot;
    out.patch_own = patch_own;
    out.patch_int = patch_int;
    out.slot_v.resize(nslot);
    out.slot_g.resize(nslot);
    out.slot_c.resize(nslot);
    for (int s = 0; s < nslot; s++) {
        int i = slot_elem[s];
        int e = eperm[i];
        const int32_t *t = m.tri + 3 * (size_t)e;
        const double *g = gph.data() + 6 * (size_t)e;
        double h0 = (m.depth[t[0]] + m.depth[t[1]] + m.depth[t[2]]) / 3.0;
        out.slot_v[s] = make_int4(vinv[t[0]], vinv[t[1]], vinv[t[2]], slot_guest[s] ? -1 - i : i);
        out.slot_g[s] = make_float4((float)g[0], (float)g[1], (float)g[2], (float)g[3]);
        out.slot_c[s] = make_float4((float)A[e], (float)h0, (float)m.coriolis[e], 0.0f);
    }

    // ---- per-vertex incidence (local slot, corner), grouped by vertex. Within a vertex the
    // entries are ordered by the caller's element id, so that the sum of a vertex's corner
    // fluxes runs in the same order whatever the patch layout: a mesh then gives bitwise
    // the same result in every execution mode, patch size and batch it is uploaded in.
    {
        std::vector<int> cnt(nv + 1, 0);
        for (int p = 0; p < npatch; p++)
            for (int s = patch_slot[p]; s < patch_slot[p + 1]; s++) {
                const int4 c = out.slot_v[s];
                int cv[3] = {c.x, c.y, c.z};
                for (int k = 0; k < 3; k++)
                    if (vpatch[cv[k]] == p) cnt[cv[k] + 1]++;
            }
        for (int v = 0; v < nv; v++) cnt[v + 1] += cnt[v];
        out.vcsr_off = cnt;
        out.vcsr.resize(cnt[nv]);
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int p = 0; p < npatch; p++)
            for (int s = patch_slot[p]; s < patch_slot[p + 1]; s++) {
                const int4 c = out.slot_v[s];
                int cv[3] = {c.x, c.y, c.z};
                for (int k = 0; k < 3; k++)
                    if (vpatch[cv[k]] == p)
                        out.vcsr[fill[cv[k]]++] = ((uint32_t)(s - patch_slot[p]) << 2) | (uint32_t)k;
            }
        auto caller_elem = [&](int v, uint32_t q) {
            const int w = out.slot_v[patch_slot[vpatch[v]] + (int)(q >> 2)].w;
            return eperm[w >= 0 ? w : -1 - w];
        };
        for (int v = 0; v < nv; v++)
            std::sort(out.vcsr.begin() + cnt[v], out.vcsr.begin() + cnt[v + 1],
                      [&](uint32_t a, uint32_t b) { return caller_elem(v, a) < caller_elem(v, b); });
    }

    out.inv_av.resize(nv);
    out.area_v.resize(nv);
    out.h0_v.resize(nv);
    for (int i = 0; i < nv; i++) {
        out.area_v[i] = Av[vperm[i]];
        out.inv_av[i] = (float)(1.0 / Av[vperm[i]]);
        out.h0_v[i] = (float)m.depth[vperm[i]];
    }
    out.area_e.resize(ne);
    out.h0_e.resize(ne);
    double gmax = 0.0;
    for (int i = 0; i < ne; i++) {
        int e = eperm[i];
        const int32_t *t = m.tri + 3 * (size_t)e;
        out.area_e[i] = A[e];
        out.h0_e[i] = (m.depth[t[0]] + m.depth[t[1]] + m.depth[t[2]]) / 3.0;
        // largest eigenvalue of the 2x2 matrix sum_k dphi_k dphi_k^T
        const double *g = gph.data() + 6 * (size_t)e;
        double sxx = 0, sxy = 0, syy = 0;
        for (int k = 0; k < 3; k++) {
            sxx += g[2 * k] * g[2 * k];
            sxy += g[2 * k] * g[2 * k + 1];
            syy += g[2 * k + 1] * g[2 * k + 1];
        }
        double tr = sxx + syy, det = sxx * syy - sxy * sxy;
        double lmax = 0.5 * tr + sqrt(std::max(0.25 * tr * tr - det, 0.0));
        gmax = std::max(gmax, out.h0_e[i] * lmax);
    }
    // Two upper bounds of lambda_max(-div H0 grad) for the lumped operator (times g
    // gives the largest squared substep frequency over dt^2): element by element,
    // max_e 3 H0_e lambda_max(sum_k dphi_k dphi_k^T), and Gershgorin over the rows of
    // K / A_v. Both are rigorous; the smaller one is kept.
    double gersh = 0.0;
    for (int v = 0; v < nv; v++) gersh = std::max(gersh, (kdiag[v] + koff[v]) / Av[v]);
    out.grad_gram_max_h = std::min(3.0 * gmax, gersh);

    // ---- neighbours across edges and the two-point flux geometry of the barotropic
    // viscosity (Eq. viscosity_BT): for edge k of an element (corner k to corner k+1)
    // with a neighbour, the neighbour, its corner opposite the edge, the rotation from
    // the neighbour's frame into this one, L/d and L^2/d (L: edge length, the mean of its
    // lengths in the two frames; d: centroid distance in the plane unfolded across the
    // edge).
    out.visc_nb.resize(ne);
    out.visc_opp.resize(ne);
    out.visc_geo.resize(3 * (size_t)ne);
    out.visc_rot = false;
    double vstiff = 0.0;
    for (int i = 0; i < ne; i++) {
        const int e = eperm[i];
        const int32_t *t = m.tri + 3 * (size_t)e;
        int nbn[3], opp[3];
        double srow = 0.0;
        for (int k = 0; k < 3; k++) {
            const int o = nb_c[3 * (size_t)e + k];
            nbn[k] = o < 0 ? -1 : einv[o];
            opp[k] = -1;
            out.visc_geo[3 * (size_t)i + k] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
            if (o < 0) continue;
            const int va = t[k], vb = t[(k + 1) % 3];
            const int32_t *to = m.tri + 3 * (size_t)o;
            int oa = 0, ob = 0;
            for (int c = 0; c < 3; c++) {
                if (to[c] == va) oa = c;
                if (to[c] == vb) ob = c;
            }
            opp[k] = vinv[to[3 - oa - ob]];
            double ang[2], along[2], perp[2], len[2];
            const int el[2] = {e, o}, ca[2] = {k, oa}, cb[2] = {(k + 1) % 3, ob};
            for (int side = 0; side < 2; side++) {
                const double *p = m.xy + 6 * (size_t)el[side];
                const double ax = p[2 * ca[side]], ay = p[2 * ca[side] + 1];
                const double ex = p[2 * cb[side]] - ax, ey = p[2 * cb[side] + 1] - ay;
                const double cx = (p[0] + p[2] + p[4]) / 3.0 - ax, cy = (p[1] + p[3] + p[5]) / 3.0 - ay;
                len[side] = std::sqrt(ex * ex + ey * ey);
                ang[side] = std::atan2(ey, ex);
                along[side] = (cx * ex + cy * ey) / len[side];
                perp[side] = std::fabs(cx * ey - cy * ex) / len[side];
            }
            const double L = 0.5 * (len[0] + len[1]);
            const double da = along[0] - along[1], dp = perp[0] + perp[1];
            const double d = std::sqrt(da * da + dp * dp);
            const double rot = ang[0] - ang[1];
            const float cr = (float)std::cos(rot), sr = (float)std::sin(rot);
            // frames that agree up to rounding (planar meshes, periodic unwrapping) count as
            // the identity: a turn below 1e-7 rad is below the FP32 rounding of the velocities
            if (!(cr == 1.0f && std::fabs(sr) < 1e-7f)) out.visc_rot = true;
            out.visc_geo[3 * (size_t)i + k] = make_float4(cr, sr, (float)(L / d), (float)(L * L / d));
            const double ho = (m.depth[to[0]] + m.depth[to[1]] + m.depth[to[2]]) / 3.0;
            srow += 0.5 * (out.h0_e[i] + ho) / out.h0_e[i] * (L / d);
        }
        out.visc_nb[i] = make_int4(nbn[0], nbn[1], nbn[2], 0);
        out.visc_opp[i] = make_int4(opp[0], opp[1], opp[2], 0);
        vstiff = std::max(vstiff, 2.0 * srow / out.area_e[i]);
    }
    out.visc_stiffness = vstiff;
    out.nbasin = 1;
    out.patch_basin.assign(npatch, 0);
    out.basin_v = {0, nv};
    out.basin_e = {0, ne};
    out.basin_patch = {0, npatch};
    out.basin_stiffness = {out.grad_gram_max_h};
    out.basin_visc_stiffness = {out.visc_stiffness};
    return SESW_OK;
}

void concat_meshes(std::vector<HostMesh> &parts, HostMesh &out)
{
    out = HostMesh();
    int nv = 0, ne = 0, np = 0, ns = 0, ncsr = 0;
    for (auto &h : parts) {
        nv += h.nv;
        ne += h.ne;
        np += h.npatch;
        ns += h.nslot;
        ncsr += (int)h.vcsr.size();
    }
    out.nv = nv;
    out.ne = ne;
    out.npatch = np;
    out.nslot = ns;
    out.nbasin = (int)parts.size();
    out.vperm.reserve(nv);
    out.eperm.reserve(ne);
    out.patch_v.assign(1, 0);
    out.patch_slot.assign(1, 0);
    out.vcsr_off.assign(1, 0);
    out.basin_v.assign(1, 0);
    out.basin_e.assign(1, 0);
    out.basin_patch.assign(1, 0);
    out.slot_v.reserve(ns);
    out.slot_g.reserve(ns);
    out.slot_c.reserve(ns);
    out.vcsr.reserve(ncsr);
    int vo = 0, eo = 0, po = 0, so = 0, co = 0;
    for (size_t b = 0; b < parts.size(); b++) {
        HostMesh &h = parts[b];
        for (int v : h.vperm) out.vperm.push_back(v + vo);
        for (int e : h.eperm) out.eperm.push_back(e + eo);
        for (int p = 1; p <= h.npatch; p++) {
            out.patch_v.push_back(h.patch_v[p] + vo);
            out.patch_slot.push_back(h.patch_slot[p] + so);
        }
        out.patch_own.insert(out.patch_own.end(), h.patch_own.begin(), h.patch_own.end());
        out.patch_int.insert(out.patch_int.end(), h.patch_int.begin(), h.patch_int.end());
        for (int p = 0; p < h.npatch; p++) out.patch_basin.push_back((int)b);
        for (const int4 &c : h.slot_v)
            out.slot_v.push_back(make_int4(c.x + vo, c.y + vo, c.z + vo, c.w >= 0 ? c.w + eo : c.w - eo));
        out.slot_g.insert(out.slot_g.end(), h.slot_g.begin(), h.slot_g.end());
        out.slot_c.insert(out.slot_c.end(), h.slot_c.begin(), h.slot_c.end());
        for (int v = 1; v <= h.nv; v++) out.vcsr_off.push_back(h.vcsr_off[v] + co);
        out.vcsr.insert(out.vcsr.end(), h.vcsr.begin(), h.vcsr.end());
        out.inv_av.insert(out.inv_av.end(), h.inv_av.begin(), h.inv_av.end());
        out.h0_v.insert(out.h0_v.end(), h.h0_v.begin(), h.h0_v.end());
        out.area_v.insert(out.area_v.end(), h.area_v.begin(), h.area_v.end());
        out.area_e.insert(out.area_e.end(), h.area_e.begin(), h.area_e.end());
        out.h0_e.insert(out.h0_e.end(), h.h0_e.begin(), h.h0_e.end());
        for (const int4 &q : h.visc_nb)
            out.visc_nb.push_back(make_int4(q.x < 0 ? -1 : q.x + eo, q.y < 0 ? -1 : q.y + eo,
                                            q.z < 0 ? -1 : q.z + eo, 0));
        for (const int4 &q : h.visc_opp)
            out.visc_opp.push_back(make_int4(q.x < 0 ? -1 : q.x + vo, q.y < 0 ? -1 : q.y + vo,
                                             q.z < 0 ? -1 : q.z + vo, 0));
        out.visc_geo.insert(out.visc_geo.end(), h.visc_geo.begin(), h.visc_geo.end());
        out.visc_rot = out.visc_rot || h.visc_rot;
        out.visc_stiffness = std::max(out.visc_stiffness, h.visc_stiffness);
        out.basin_visc_stiffness.push_back(h.visc_stiffness);
        out.max_patch_slots = std::max(out.max_patch_slots, h.max_patch_slots);
        out.max_patch_vertices = std::max(out.max_patch_vertices, h.max_patch_vertices);
        out.patch_vertices = std::max(out.patch_vertices, h.patch_vertices);
        out.grad_gram_max_h = std::max(out.grad_gram_max_h, h.grad_gram_max_h);
        out.basin_stiffness.push_back(h.grad_gram_max_h);
        vo += h.nv;
        eo += h.ne;
        po += h.npatch;
        so += h.nslot;
        co += (int)h.vcsr.size();
        out.basin_v.push_back(vo);
        out.basin_e.push_back(eo);
        out.basin_patch.push_back(po);
    }
}

int build_halos(HostMesh &hm, std::string &err)
{
    const int np = hm.npatch;
    hm.patch_halo.assign(np + 1, 0);
    hm.halo_v.clear();
    hm.slot_l.assign(hm.nslot, make_ushort4(0, 0, 0, 0));
    hm.max_patch_local = 0;
    hm.max_patch_halo = 0;
    hm.max_patch_csr = 0;
    std::vector<int> halo;
    for (int p = 0; p < np; p++) {
        const int vlo = hm.patch_v[p], vhi = hm.patch_v[p + 1], nown = vhi - vlo;
        halo.clear();
        for (int s = hm.patch_slot[p]; s < hm.patch_slot[p + 1]; s++) {
            const int4 c = hm.slot_v[s];
            const int cv[3] = {c.x, c.y, c.z};
            for (int k = 0; k < 3; k++)
                if (cv[k] < vlo || cv[k] >= vhi) halo.push_back(cv[k]);
        }
        std::sort(halo.begin(), halo.end());
        halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
        const int nloc = nown + (int)halo.size();
        if (nloc > 65535) {
            err = "a patch has more than 65535 local vertices; the persistent kernel needs smaller patches";
            return SESW_EINVAL;
        }
        for (int s = hm.patch_slot[p]; s < hm.patch_slot[p + 1]; s++) {
            const int4 c = hm.slot_v[s];
            const int cv[3] = {c.x, c.y, c.z};
            unsigned short l[3];
            for (int k = 0; k < 3; k++) {
                if (cv[k] >= vlo && cv[k] < vhi)
                    l[k] = (unsigned short)(cv[k] - vlo);
                else
                    l[k] = (unsigned short)(nown + (std::lower_bound(halo.begin(), halo.end(), cv[k]) - halo.begin()));
            }
            hm.slot_l[s] = make_ushort4(l[0], l[1], l[2], 0);
        }
        hm.halo_v.insert(hm.halo_v.end(), halo.begin(), halo.end());
        hm.patch_halo[p + 1] = (int)hm.halo_v.size();
        hm.max_patch_local = std::max(hm.max_patch_local, nloc);
        hm.max_patch_halo = std::max(hm.max_patch_halo, (int)halo.size());
        hm.max_patch_csr = std::max(hm.max_patch_csr, hm.vcsr_off[vhi] - hm.vcsr_off[vlo]);
    }
    return SESW_OK;
}

}  // namespace sesw
