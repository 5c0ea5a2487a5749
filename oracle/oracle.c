/*
 * FP64 CPU oracle for the split-explicit barotropic subcycle of Banerjee, Scholz,
 * Danilov, Klingbeil and Sidorenko, "Split-explicit external mode solver in finite
 * volume sea ice ocean model FESOM2" (arXiv 2311.08241).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference against which the
 * CUDA path is checked. Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it; the library never links or calls it, and it shares no code,
 * header, table or helper with the library.
 *
 * What it computes (all in double precision, no FMA contraction: build with
 * -ffp-contract=off):
 *
 *   Barotropic system, Eq. (4.5):  dU/dt + f e_z x U + g H grad(eta) = R,
 *                                  deta/dt + div(U) + W = 0,   H = H0 + eta
 *   (W = 0 except in oracle_advance_ext, which also adds the viscous regularisation
 *   of Eq. (viscosity_BT); its discretisation is described there).
 *   Substep of the dissipative forward-backward scheme, Eq. (4.10), dt = tau/M:
 *       U^{m+1} = U^m - dt [ (f/2) e_z x (U^{m+1} + U^m) + g H^m grad(eta^m) - R ]
 *       eta^{m+1} = eta^m - dt div[ (1+theta) U^{m+1} - theta U^m ]
 *     (the bracket of Eq. 4.10 is printed with "- gH grad(eta) - R"; the signs
 *      used here are the ones Eq. 4.5 fixes.)
 *   After M substeps, Sect. 2.3: <eta>^{n+1} = eta^M, <U>^{n+1} = U^M, and the
 *   time-mean transport of Eq. (4.12):
 *       <<U>> = (1/M) sum_{m=1..M} U^m + (theta/M) (U^M - U^0).
 *   U^0 of a baroclinic step is the U^M of the previous one (Sect. 2.3).
 *
 * Spatial discretisation (the paper defers it to Danilov et al. 2017): eta on
 * vertices, U constant on triangles. The gradient of eta on a triangle is the
 * Green-Gauss contour sum over its three edges (exact for the linear interpolant).
 * The divergence at a vertex is the net flux out of its median-dual cell (the
 * polygon joining edge midpoints and triangle centroids around the vertex) divided
 * by that cell's area; it is evaluated edge by edge: for an edge (a,b) each
 * adjacent triangle contributes the flux of its U through the segment from the
 * edge midpoint to the triangle centroid, counted out of a's cell and into b's.
 * A coast edge has one adjacent triangle and no flux through the coast itself.
 * H on a triangle is the mean of H0 + eta over its corners (H0 alone when the
 * linear option is chosen). Coriolis is taken at the triangle centroid.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Working precision. The oracle is built with double; a float build of the same
 * source is used only to calibrate how far FP32 arithmetic of this algorithm drifts
 * from FP64 (the parity tolerances of the FP32 GPU path). Mesh geometry (areas,
 * edge normals, dual-cell segments) is always computed in double and then stored in
 * the working precision; the time stepping uses `real` throughout; the interface
 * stays double and converts at entry and exit. */
#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;

typedef struct {
    int nv, ne, ned;
    int *tri;          /* ne*3 */
    real *nrm;         /* ne*6, outward normal times length of each triangle edge k -> k+1 */
    real *depth_v;     /* nv */
    real *f_e;         /* ne */
    real *area_e;      /* ne, shoelace area of the triangle */
    real *area_v;      /* nv, median-dual cell area */
    int *edge_v;       /* ned*2, edge_v[2k] < edge_v[2k+1] */
    int *edge_e;       /* ned*2, adjacent triangles, -1 where absent */
    real *seg;         /* ned*2*2: (Nx,Ny) per side, the segment's normal times length,
                          pointing from the cell of edge_v[2k] into that of edge_v[2k+1] */
    int *vedge_off;    /* nv+1 */
    int *vedge;        /* 2*ned, incident edges of each vertex in increasing edge order */
} omesh;

static void omesh_free(omesh *m)
{
    if (!m) return;
    free(m->tri); free(m->nrm); free(m->depth_v); free(m->f_e); free(m->area_e); free(m->area_v);
    free(m->edge_v); free(m->edge_e); free(m->seg); free(m->vedge_off); free(m->vedge);
    free(m);
}

typedef struct { long long key; int e; int k; } halfedge;

static int cmp_half(const void *pa, const void *pb)
{
    const halfedge *a = (const halfedge *)pa, *b = (const halfedge *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    if (a->e != b->e) return a->e < b->e ? -1 : 1;
    return a->k - b->k;
}

/* Polygon area by the shoelace formula, vertices in order. */
static double shoelace(const double *px, const double *py, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; i++) {
        int j = (i + 1) % n;
        s += px[i] * py[j] - px[j] * py[i];
    }
    return 0.5 * s;
}

/* Build the oracle's mesh. status: 0 ok, -1 bad index, -2 non-positive area,
 * -3 an edge shared by more than two triangles, -4 allocation. */
void *oracle_mesh_new(int nv, int ne, const int *tri, const double *xy,
                      const double *depth_v, const double *f_e, int *status)
{
    *status = 0;
    omesh *m = (omesh *)calloc(1, sizeof(omesh));
    if (!m) { *status = -4; return NULL; }
    m->nv = nv; m->ne = ne;
    m->tri = (int *)malloc(sizeof(int) * 3 * (size_t)ne);
    m->nrm = (real *)malloc(sizeof(real) * 6 * (size_t)ne);
    m->depth_v = (real *)malloc(sizeof(real) * (size_t)nv);
    m->f_e = (real *)malloc(sizeof(real) * (size_t)ne);
    m->area_e = (real *)malloc(sizeof(real) * (size_t)ne);
    m->area_v = (real *)calloc((size_t)nv, sizeof(real));
    double *av = (double *)calloc((size_t)nv, sizeof(double));
    if (!m->tri || !m->nrm || !m->depth_v || !m->f_e || !m->area_e || !m->area_v || !av) {
        free(av); *status = -4; omesh_free(m); return NULL;
    }
    memcpy(m->tri, tri, sizeof(int) * 3 * (size_t)ne);
    for (int v = 0; v < nv; v++) m->depth_v[v] = (real)depth_v[v];
    for (int e = 0; e < ne; e++) m->f_e[e] = (real)f_e[e];

    for (int e = 0; e < ne; e++)
        for (int k = 0; k < 3; k++)
            if (tri[3 * e + k] < 0 || tri[3 * e + k] >= nv) { free(av); *status = -1; omesh_free(m); return NULL; }

    /* triangle areas, edge normals and median-dual cell areas (sub-quad of each corner) */
    for (int e = 0; e < ne; e++) {
        const double *p = xy + 6 * (size_t)e;
        double px[3] = {p[0], p[2], p[4]}, py[3] = {p[1], p[3], p[5]};
        double A = shoelace(px, py, 3);
        if (!(A > 0.0)) { free(av); *status = -2; omesh_free(m); return NULL; }
        m->area_e[e] = (real)A;
        double cx = (px[0] + px[1] + px[2]) / 3.0, cy = (py[0] + py[1] + py[2]) / 3.0;
        for (int k = 0; k < 3; k++) {
            int kn = (k + 1) % 3, kp = (k + 2) % 3;
            /* outward normal times length of a counter-clockwise edge (dx,dy) is (dy,-dx) */
            m->nrm[6 * e + 2 * k] = (real)(py[kn] - py[k]);
            m->nrm[6 * e + 2 * k + 1] = (real)(-(px[kn] - px[k]));
            double qx[4] = {px[k], 0.5 * (px[k] + px[kn]), cx, 0.5 * (px[k] + px[kp])};
            double qy[4] = {py[k], 0.5 * (py[k] + py[kn]), cy, 0.5 * (py[k] + py[kp])};
            av[tri[3 * e + k]] += shoelace(qx, qy, 4);
        }
    }
    for (int v = 0; v < nv; v++) m->area_v[v] = (real)av[v];
    free(av);

    /* edges: group the 3*ne half-edges by their unordered vertex pair */
    halfedge *h = (halfedge *)malloc(sizeof(halfedge) * 3 * (size_t)ne);
    if (!h) { *status = -4; omesh_free(m); return NULL; }
    for (int e = 0; e < ne; e++)
        for (int k = 0; k < 3; k++) {
            long long a = tri[3 * e + k], b = tri[3 * e + (k + 1) % 3];
            long long lo = a < b ? a : b, hi = a < b ? b : a;
            h[3 * e + k].key = lo * (long long)nv + hi;
            h[3 * e + k].e = e;
            h[3 * e + k].k = k;
        }
    qsort(h, 3 * (size_t)ne, sizeof(halfedge), cmp_half);
    int ned = 0;
    for (size_t i = 0; i < 3 * (size_t)ne;) {
        size_t j = i;
        while (j < 3 * (size_t)ne && h[j].key == h[i].key) j++;
        if (j - i > 2) { free(h); *status = -3; omesh_free(m); return NULL; }
        ned++;
        i = j;
    }
    m->ned = ned;
    m->edge_v = (int *)malloc(sizeof(int) * 2 * (size_t)ned);
    m->edge_e = (int *)malloc(sizeof(int) * 2 * (size_t)ned);
    m->seg = (real *)calloc(4 * (size_t)ned, sizeof(real));
    if (!m->edge_v || !m->edge_e || !m->seg) { free(h); *status = -4; omesh_free(m); return NULL; }
    int k = 0;
    for (size_t i = 0; i < 3 * (size_t)ne;) {
        size_t j = i;
        while (j < 3 * (size_t)ne && h[j].key == h[i].key) j++;
        int a = (int)(h[i].key / nv), b = (int)(h[i].key % nv);
        m->edge_v[2 * k] = a;
        m->edge_v[2 * k + 1] = b;
        m->edge_e[2 * k] = -1;
        m->edge_e[2 * k + 1] = -1;
        for (size_t s = i; s < j; s++) {
            int e = h[s].e;
            int side = (int)(s - i);
            m->edge_e[2 * k + side] = e;
            /* corners of a and b inside e */
            const double *p = xy + 6 * (size_t)e;
            int ka = -1, kb = -1;
            for (int c = 0; c < 3; c++) {
                if (tri[3 * e + c] == a) ka = c;
                if (tri[3 * e + c] == b) kb = c;
            }
            double ax = p[2 * ka], ay = p[2 * ka + 1], bx = p[2 * kb], by = p[2 * kb + 1];
            double cx = (p[0] + p[2] + p[4]) / 3.0, cy = (p[1] + p[3] + p[5]) / 3.0;
            double mx = 0.5 * (ax + bx), my = 0.5 * (ay + by);
            double dx = cx - mx, dy = cy - my;
            double nx = dy, ny = -dx;               /* one of the two normals of length |d| */
            if (nx * (bx - ax) + ny * (by - ay) < 0.0) { nx = -nx; ny = -ny; }
            m->seg[4 * k + 2 * side] = (real)nx;
            m->seg[4 * k + 2 * side + 1] = (real)ny;
        }
        k++;
        i = j;
    }
    free(h);

    /* incident edges per vertex, for an ordered per-vertex sum */
    m->vedge_off = (int *)calloc((size_t)nv + 1, sizeof(int));
    m->vedge = (int *)malloc(sizeof(int) * 2 * (size_t)ned);
    if (!m->vedge_off || !m->vedge) { *status = -4; omesh_free(m); return NULL; }
    for (int q = 0; q < ned; q++) {
        m->vedge_off[m->edge_v[2 * q] + 1]++;
        m->vedge_off[m->edge_v[2 * q + 1] + 1]++;
    }
    for (int v = 0; v < nv; v++) m->vedge_off[v + 1] += m->vedge_off[v];
    int *fill = (int *)malloc(sizeof(int) * (size_t)nv);
    if (!fill) { *status = -4; omesh_free(m); return NULL; }
    memcpy(fill, m->vedge_off, sizeof(int) * (size_t)nv);
    for (int q = 0; q < ned; q++) {
        m->vedge[fill[m->edge_v[2 * q]]++] = q;
        m->vedge[fill[m->edge_v[2 * q + 1]]++] = q;
    }
    free(fill);
    return m;
}

void oracle_mesh_free(void *hm) { omesh_free((omesh *)hm); }

int oracle_mesh_info(void *hm, int *ned, int *nbnd)
{
    omesh *m = (omesh *)hm;
    int nb = 0;
    for (int q = 0; q < m->ned; q++) nb += (m->edge_e[2 * q + 1] < 0);
    *ned = m->ned;
    *nbnd = nb;
    return 0;
}

int oracle_areas(void *hm, double *area_v, double *area_e)
{
    omesh *m = (omesh *)hm;
    if (area_v) for (int v = 0; v < m->nv; v++) area_v[v] = (double)m->area_v[v];
    if (area_e) for (int e = 0; e < m->ne; e++) area_e[e] = (double)m->area_e[e];
    return 0;
}

int oracle_edges(void *hm, int *edge_v, int *edge_e)
{
    omesh *m = (omesh *)hm;
    memcpy(edge_v, m->edge_v, sizeof(int) * 2 * (size_t)m->ned);
    memcpy(edge_e, m->edge_e, sizeof(int) * 2 * (size_t)m->ned);
    return 0;
}

/* Green-Gauss gradient of the vertex field eta on triangle e. */
static void gradient_e(const omesh *m, int e, const real *eta, real *gx, real *gy)
{
    const real *n = m->nrm + 6 * e;
    const int *t = m->tri + 3 * e;
    real sx = 0, sy = 0;
    for (int k = 0; k < 3; k++) {
        int kn = (k + 1) % 3;
        real etam = (eta[t[k]] + eta[t[kn]]) / 2;
        sx += etam * n[2 * k];
        sy += etam * n[2 * k + 1];
    }
    *gx = sx / m->area_e[e];
    *gy = sy / m->area_e[e];
}

int oracle_gradient(void *hm, const double *eta, double *grad)
{
    omesh *m = (omesh *)hm;
    real *er = (real *)malloc(sizeof(real) * (size_t)m->nv);
    if (!er) return -4;
    for (int v = 0; v < m->nv; v++) er[v] = (real)eta[v];
    for (int e = 0; e < m->ne; e++) {
        real gx, gy;
        gradient_e(m, e, er, &gx, &gy);
        grad[2 * e] = (double)gx;
        grad[2 * e + 1] = (double)gy;
    }
    free(er);
    return 0;
}

/* Net outflow of F through the median-dual cell boundary of every vertex, per area. */
static void divergence(const omesh *m, const real *F, real *edgeflux, real *div)
{
    int ned = m->ned, nv = m->nv;
    #pragma omp parallel for schedule(static)
    for (int q = 0; q < ned; q++) {
        real s = 0;
        for (int side = 0; side < 2; side++) {
            int e = m->edge_e[2 * q + side];
            if (e < 0) continue;
            s += F[2 * e] * m->seg[4 * q + 2 * side] + F[2 * e + 1] * m->seg[4 * q + 2 * side + 1];
        }
        edgeflux[q] = s;     /* out of edge_v[2q], into edge_v[2q+1] */
    }
    #pragma omp parallel for schedule(static)
    for (int v = 0; v < nv; v++) {
        real s = 0;
        for (int i = m->vedge_off[v]; i < m->vedge_off[v + 1]; i++) {
            int q = m->vedge[i];
            s += (m->edge_v[2 * q] == v) ? edgeflux[q] : -edgeflux[q];
        }
        div[v] = s / m->area_v[v];
    }
}

int oracle_divergence(void *hm, const double *F, double *div)
{
    omesh *m = (omesh *)hm;
    real *ef = (real *)malloc(sizeof(real) * (size_t)m->ned);
    real *Fr = (real *)malloc(sizeof(real) * 2 * (size_t)m->ne);
    real *dr = (real *)malloc(sizeof(real) * (size_t)m->nv);
    if (!ef || !Fr || !dr) { free(ef); free(Fr); free(dr); return -4; }
    for (size_t i = 0; i < 2 * (size_t)m->ne; i++) Fr[i] = (real)F[i];
    divergence(m, Fr, ef, dr);
    for (int v = 0; v < m->nv; v++) div[v] = (double)dr[v];
    free(ef); free(Fr); free(dr);
    return 0;
}

static real element_depth(const omesh *m, int e, const real *eta, int nonlinear_h)
{
    const int *t = m->tri + 3 * e;
    real H = (m->depth_v[t[0]] + m->depth_v[t[1]] + m->depth_v[t[2]]) / 3;
    if (nonlinear_h) H += (eta[t[0]] + eta[t[1]] + eta[t[2]]) / 3;
    return H;
}

/* Volume sum A_v eta_v and energy sum A_v g eta^2/2 + sum A_e |U|^2/(2 H_e), in double. */
int oracle_diagnostics(void *hm, const double *eta, const double *U, double g, int nonlinear_h,
                       double *volume, double *energy)
{
    omesh *m = (omesh *)hm;
    double vol = 0.0, en = 0.0;
    for (int v = 0; v < m->nv; v++) {
        vol += (double)m->area_v[v] * eta[v];
        en += (double)m->area_v[v] * 0.5 * g * eta[v] * eta[v];
    }
    for (int e = 0; e < m->ne; e++) {
        const int *t = m->tri + 3 * e;
        double H = ((double)m->depth_v[t[0]] + (double)m->depth_v[t[1]] + (double)m->depth_v[t[2]]) / 3.0;
        if (nonlinear_h) H += (eta[t[0]] + eta[t[1]] + eta[t[2]]) / 3.0;
        en += (double)m->area_e[e] * (U[2 * e] * U[2 * e] + U[2 * e + 1] * U[2 * e + 1]) / (2.0 * H);
    }
    *volume = vol;
    *energy = en;
    return 0;
}

/*
 * Advance nsteps baroclinic steps of the SE subcycle.
 *   R      ne*2 frozen forcing (element frame, m^2/s^2)
 *   eta    nv, in: <eta>^n, out: <eta>^{n+nsteps}
 *   U      ne*2, in: U^0 of the first step (the carried <U>^n), out: U^M of the last
 *   Umean  ne*2, out: <<U>> of the last step (Eq. 4.12)
 *   diag   NULL or nsteps*2: (volume, energy) after each step
 *   eta_mean_out  NULL or nv: (1/M) sum_{m=0..M-1} eta^m of the last step
 * Returns 0, or -4 on allocation failure, -5 if M < 1.
 */
int oracle_advance(void *hm, const double *R_in, double g_in, double theta_in, double tau, int M,
                   int nonlinear_h, int nsteps, double *eta_io, double *U_io, double *Umean_out, double *diag,
                   double *eta_mean_out)
{
    omesh *m = (omesh *)hm;
    if (M < 1) return -5;
    int ne = m->ne, nv = m->nv;
    const real dt = (real)(tau / (double)M);
    const real g = (real)g_in, theta = (real)theta_in;
    real *F = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *U = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *U0 = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *sumU = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *R = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *eta = (real *)malloc(sizeof(real) * (size_t)nv);
    real *div = (real *)malloc(sizeof(real) * (size_t)nv);
    real *ef = (real *)malloc(sizeof(real) * (size_t)m->ned);
    double *Ud = (double *)malloc(sizeof(double) * 2 * (size_t)ne);
    if (!F || !U || !U0 || !sumU || !R || !eta || !div || !ef || !Ud) {
        free(F); free(U); free(U0); free(sumU); free(R); free(eta); free(div); free(ef); free(Ud);
        return -4;
    }
    for (size_t i = 0; i < 2 * (size_t)ne; i++) { U[i] = (real)U_io[i]; R[i] = (real)R_in[i]; }
    for (int v = 0; v < nv; v++) eta[v] = (real)eta_io[v];
    for (int n = 0; n < nsteps; n++) {
        memcpy(U0, U, sizeof(real) * 2 * (size_t)ne);
        memset(sumU, 0, sizeof(real) * 2 * (size_t)ne);
        if (eta_mean_out)
            for (int v = 0; v < nv; v++) eta_mean_out[v] = 0.0;
        for (int s = 0; s < M; s++) {
            if (eta_mean_out)
                for (int v = 0; v < nv; v++) eta_mean_out[v] += (double)eta[v] / (double)M;
            /* momentum: Crank-Nicolson Coriolis, pressure at eta^m with H^m, frozen R */
            #pragma omp parallel for schedule(static)
            for (int e = 0; e < ne; e++) {
                real gx, gy;
                gradient_e(m, e, eta, &gx, &gy);
                real H = element_depth(m, e, eta, nonlinear_h);
                real a = dt * m->f_e[e] / 2;
                real ux = U[2 * e], uy = U[2 * e + 1];
                /* (I + a J) U' = (I - a J) U + dt (-g H grad eta + R),  J = [[0,-1],[1,0]] */
                real A11 = 1, A12 = -a, A21 = a, A22 = 1;
                real bx = ux + a * uy + dt * (-g * H * gx + R[2 * e]);
                real by = -a * ux + uy + dt * (-g * H * gy + R[2 * e + 1]);
                real det = A11 * A22 - A12 * A21;
                real nx = (bx * A22 - A12 * by) / det;
                real ny = (A11 * by - A21 * bx) / det;
                F[2 * e] = (1 + theta) * nx - theta * ux;
                F[2 * e + 1] = (1 + theta) * ny - theta * uy;
                U[2 * e] = nx;
                U[2 * e + 1] = ny;
                sumU[2 * e] += nx;
                sumU[2 * e + 1] += ny;
            }
            /* continuity with the theta-weighted transport */
            divergence(m, F, ef, div);
            #pragma omp parallel for schedule(static)
            for (int v = 0; v < nv; v++) eta[v] -= dt * div[v];
        }
        for (int e = 0; e < ne; e++)
            for (int c = 0; c < 2; c++)
                Umean_out[2 * e + c] = (double)(sumU[2 * e + c] / (real)M + theta / (real)M * (U[2 * e + c] - U0[2 * e + c]));
        if (diag) {
            double *ed = (double *)malloc(sizeof(double) * (size_t)nv);
            if (ed) {
                for (int v = 0; v < nv; v++) ed[v] = (double)eta[v];
                for (size_t i = 0; i < 2 * (size_t)ne; i++) Ud[i] = (double)U[i];
                oracle_diagnostics(m, ed, Ud, g_in, nonlinear_h, diag + 2 * n, diag + 2 * n + 1);
                free(ed);
            }
        }
    }
    for (size_t i = 0; i < 2 * (size_t)ne; i++) U_io[i] = (double)U[i];
    for (int v = 0; v < nv; v++) eta_io[v] = (double)eta[v];
    free(F); free(U); free(U0); free(sumU); free(R); free(eta); free(div); free(ef); free(Ud);
    return 0;
}

/*
 * Advance nsteps baroclinic steps of the AB3-AM4 substep with dissipative coefficients
 * (SESM), Eqs. (4.7)-(4.8), with the freshwater flux W (NULL: W = 0):
 *     U_AB   = (3/2 + beta) U^m - (1/2 + 2 beta) U^{m-1} + beta U^{m-2}
 *     eta^{m+1} = eta^m - dt (div(U_AB) + W)
 *     eta_AM = delta eta^{m+1} + (1 - delta - gamma - zeta) eta^m + gamma eta^{m-1} + zeta eta^{m-2}
 *     U^{m+1} = U^m + dt ( -f e_z x U_AB - g H_AM grad(eta_AM) + R ),  H_AM = H0 + eta_AM
 *                                                    (H0 alone when nonlinear_h = 0)
 * Levels before the start of the subcycle (m - k < 0) are taken equal to level 0.
 * The time-mean transport is the mean of the transports the continuity equation used,
 *     <<U>> = (1/M) sum_{m=0..M-1} U_AB^m,
 * which makes eta^M - eta^0 = -tau (div <<U>> + W) exact (Eq. 4.11).
 */
static int advance_sesm(void *hm, const double *R_in, const double *W_in, double g_in, double beta_in,
                        double delta_in, double gamma_in, double zeta_in, double tau, int M, int nonlinear_h,
                        int nsteps, double *eta_io, double *U_io, double *Umean_out)
{
    omesh *m = (omesh *)hm;
    if (M < 1) return -5;
    const int ne = m->ne, nv = m->nv;
    const real dt = (real)(tau / (double)M);
    const real g = (real)g_in, beta = (real)beta_in, delta = (real)delta_in, gam = (real)gamma_in,
               zeta = (real)zeta_in;
    const real ab0 = (real)1.5 + beta, ab1 = -((real)0.5 + 2 * beta), ab2 = beta;
    const real am0 = delta, am1 = 1 - delta - gam - zeta, am2 = gam, am3 = zeta;
    real *U[3], *E[4];
    for (int k = 0; k < 3; k++) U[k] = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    for (int k = 0; k < 4; k++) E[k] = (real *)malloc(sizeof(real) * (size_t)nv);
    real *UAB = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *sumF = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *R = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *eAM = (real *)malloc(sizeof(real) * (size_t)nv);
    real *div = (real *)malloc(sizeof(real) * (size_t)nv);
    real *ef = (real *)malloc(sizeof(real) * (size_t)m->ned);
    real *W = (real *)calloc((size_t)nv, sizeof(real));
    int ok = UAB && sumF && R && eAM && div && ef && W;
    for (int k = 0; k < 3; k++) ok = ok && U[k];
    for (int k = 0; k < 4; k++) ok = ok && E[k];
    if (!ok) {
        for (int k = 0; k < 3; k++) free(U[k]);
        for (int k = 0; k < 4; k++) free(E[k]);
        free(UAB); free(sumF); free(R); free(eAM); free(div); free(ef); free(W);
        return -4;
    }
    for (size_t i = 0; i < 2 * (size_t)ne; i++) { U[0][i] = (real)U_io[i]; R[i] = (real)R_in[i]; }
    for (int v = 0; v < nv; v++) { E[0][v] = (real)eta_io[v]; if (W_in) W[v] = (real)W_in[v]; }
    for (int n = 0; n < nsteps; n++) {
        /* U[0] = U^m, U[1] = U^{m-1}, U[2] = U^{m-2}; E[0] = eta^m, E[1..3] older levels */
        memcpy(U[1], U[0], sizeof(real) * 2 * (size_t)ne);
        memcpy(U[2], U[0], sizeof(real) * 2 * (size_t)ne);
        for (int k = 1; k < 4; k++) memcpy(E[k], E[0], sizeof(real) * (size_t)nv);
        memset(sumF, 0, sizeof(real) * 2 * (size_t)ne);
        for (int s = 0; s < M; s++) {
            for (size_t i = 0; i < 2 * (size_t)ne; i++) {
                UAB[i] = ab0 * U[0][i] + ab1 * U[1][i] + ab2 * U[2][i];
                sumF[i] += UAB[i];
            }
            /* continuity with the AB3 transport: eta^{m+1} into the oldest level's array */
            divergence(m, UAB, ef, div);
            real *enew = E[3];
            for (int v = 0; v < nv; v++) enew[v] = E[0][v] - dt * (div[v] + W[v]);
            /* AM4 elevation: eta^{m+1}, eta^m, eta^{m-1}, eta^{m-2} */
            for (int v = 0; v < nv; v++) eAM[v] = am0 * enew[v] + am1 * E[0][v] + am2 * E[1][v] + am3 * E[2][v];
            /* momentum with explicit Coriolis on U_AB and the AM4 pressure gradient; U^{m+1}
               goes into the array of U^{m-2}, which is no longer needed */
            real *unew = U[2];
            #pragma omp parallel for schedule(static)
            for (int e = 0; e < ne; e++) {
                real gx, gy;
                gradient_e(m, e, eAM, &gx, &gy);
                real H = element_depth(m, e, eAM, nonlinear_h);
                real ux = UAB[2 * e], uy = UAB[2 * e + 1];
                /* -f e_z x U_AB = (f U_AB_y, -f U_AB_x) */
                unew[2 * e] = U[0][2 * e] + dt * (m->f_e[e] * uy - g * H * gx + R[2 * e]);
                unew[2 * e + 1] = U[0][2 * e + 1] + dt * (-m->f_e[e] * ux - g * H * gy + R[2 * e + 1]);
            }
            /* rotate the levels */
            real *t = U[2]; U[2] = U[1]; U[1] = U[0]; U[0] = t;
            real *te = E[3]; E[3] = E[2]; E[2] = E[1]; E[1] = E[0]; E[0] = te;
        }
        for (size_t i = 0; i < 2 * (size_t)ne; i++) Umean_out[i] = (double)(sumF[i] / (real)M);
    }
    for (size_t i = 0; i < 2 * (size_t)ne; i++) U_io[i] = (double)U[0][i];
    for (int v = 0; v < nv; v++) eta_io[v] = (double)E[0][v];
    for (int k = 0; k < 3; k++) free(U[k]);
    for (int k = 0; k < 4; k++) free(E[k]);
    free(UAB); free(sumF); free(R); free(eAM); free(div); free(ef); free(W);
    return 0;
}

int oracle_advance_sesm(void *hm, const double *R_in, double g_in, double beta_in, double delta_in,
                        double gamma_in, double zeta_in, double tau, int M, int nonlinear_h, int nsteps,
                        double *eta_io, double *U_io, double *Umean_out)
{
    return advance_sesm(hm, R_in, NULL, g_in, beta_in, delta_in, gamma_in, zeta_in, tau, M, nonlinear_h, nsteps,
                        eta_io, U_io, Umean_out);
}

int oracle_advance_sesm_w(void *hm, const double *R_in, const double *W_in, double g_in, double beta_in,
                          double delta_in, double gamma_in, double zeta_in, double tau, int M, int nonlinear_h,
                          int nsteps, double *eta_io, double *U_io, double *Umean_out)
{
    return advance_sesm(hm, R_in, W_in, g_in, beta_in, delta_in, gamma_in, zeta_in, tau, M, nonlinear_h, nsteps,
                        eta_io, U_io, Umean_out);
}

/*
 * Barotropic viscous regularisation R_hV = div( H A grad(U/H) ) (Eq. viscosity_BT), edge by
 * edge: for an interior edge of length L between triangles e1 and e2 with centroid
 * distance d (measured in the plane unfolded across the edge; L is the mean of the edge's
 * length in the two element frames), velocities u = U/H on
 * the triangles, and u2' = u2 rotated into e1's frame (the rotation that maps the
 * edge direction of e2's frame onto that of e1's frame),
 *     flux into e1 = H_edge A_edge (u2' - u1) L / d,   H_edge = (H1 + H2)/2,
 *     A_edge = A_bg + C_v |u2' - u1| L,
 * added to e1 divided by A_e1, and the opposite flux (rotated back) to e2. Coast edges
 * carry no flux (free slip). H is H0 (+ corner-mean eta when nonlinear).
 */
static void viscosity(const omesh *m, const real *U, const real *eta, int nonlinear_h, real Abg, real Cv,
                      const double *xy, real *out)
{
    memset(out, 0, sizeof(real) * 2 * (size_t)m->ne);
    for (int q = 0; q < m->ned; q++) {
        const int e1 = m->edge_e[2 * q], e2 = m->edge_e[2 * q + 1];
        if (e1 < 0 || e2 < 0) continue;
        const int a = m->edge_v[2 * q], b = m->edge_v[2 * q + 1];
        double geo[2][4];       /* per side: edge angle, along-edge centroid coordinate, height, edge length */
        const int es[2] = {e1, e2};
        for (int side = 0; side < 2; side++) {
            const int e = es[side];
            const double *p = xy + 6 * (size_t)e;
            int ka = 0, kb = 0;
            for (int c = 0; c < 3; c++) {
                if (m->tri[3 * e + c] == a) ka = c;
                if (m->tri[3 * e + c] == b) kb = c;
            }
            const double ax = p[2 * ka], ay = p[2 * ka + 1], bx = p[2 * kb], by = p[2 * kb + 1];
            const double cx = (p[0] + p[2] + p[4]) / 3.0, cy = (p[1] + p[3] + p[5]) / 3.0;
            const double ex = bx - ax, ey = by - ay, len = sqrt(ex * ex + ey * ey);
            geo[side][0] = atan2(ey, ex);
            geo[side][1] = ((cx - ax) * ex + (cy - ay) * ey) / len;
            geo[side][2] = fabs((cx - ax) * ey - (cy - ay) * ex) / len;
            geo[side][3] = len;
        }
        const double L = 0.5 * (geo[0][3] + geo[1][3]);   /* the two frames may differ slightly (sphere) */
        const double d = sqrt((geo[0][1] - geo[1][1]) * (geo[0][1] - geo[1][1]) +
                              (geo[0][2] + geo[1][2]) * (geo[0][2] + geo[1][2]));
        const double rot = geo[0][0] - geo[1][0];     /* from e2's frame to e1's frame */
        const real cr = (real)cos(rot), sr = (real)sin(rot);
        const real H1 = element_depth(m, e1, eta, nonlinear_h), H2 = element_depth(m, e2, eta, nonlinear_h);
        const real u1x = U[2 * e1] / H1, u1y = U[2 * e1 + 1] / H1;
        const real v2x = U[2 * e2] / H2, v2y = U[2 * e2 + 1] / H2;
        const real u2x = cr * v2x - sr * v2y, u2y = sr * v2x + cr * v2y;
        const real dx = u2x - u1x, dy = u2y - u1y;
        const real A = Abg + Cv * (real)sqrt((double)(dx * dx + dy * dy)) * (real)L;
        const real k = (H1 + H2) / 2 * A * (real)(L / d);
        const real fx = k * dx, fy = k * dy;                   /* into e1, e1's frame */
        out[2 * e1] += fx / m->area_e[e1];
        out[2 * e1 + 1] += fy / m->area_e[e1];
        /* into e2: the opposite flux rotated back into e2's frame */
        out[2 * e2] += (-(cr * fx + sr * fy)) / m->area_e[e2];
        out[2 * e2 + 1] += (-(-sr * fx + cr * fy)) / m->area_e[e2];
    }
}

int oracle_viscosity(void *hm, const double *xy, const double *U_in, const double *eta_in, int nonlinear_h,
                     double Abg, double Cv, double *out)
{
    omesh *m = (omesh *)hm;
    real *U = (real *)calloc(2 * (size_t)m->ne, sizeof(real));
    real *eta = (real *)calloc((size_t)m->nv, sizeof(real));
    real *o = (real *)calloc(2 * (size_t)m->ne, sizeof(real));
    if (!U || !eta || !o) { free(U); free(eta); free(o); return -4; }
    for (size_t i = 0; i < 2 * (size_t)m->ne; i++) U[i] = (real)U_in[i];
    for (int v = 0; v < m->nv; v++) eta[v] = (real)eta_in[v];
    viscosity(m, U, eta, nonlinear_h, (real)Abg, (real)Cv, xy, o);
    for (size_t i = 0; i < 2 * (size_t)m->ne; i++) out[i] = (double)o[i];
    free(U); free(eta); free(o);
    return 0;
}

/*
 * SE steps (as oracle_advance) with the two optional terms of Eq. (4.5) and
 * Eq. (viscosity_BT): the freshwater flux W (m/s per vertex, positive out of the ocean),
 *     eta^{m+1} = eta^m - dt ( div[(1+theta) U^{m+1} - theta U^m] + W ),
 * and the viscous regularisation added to the forcing as R + R_hV(U^m) - R_hV(U^0)
 * (its value at the start of the step subtracted, Sect. 2.2), H of R_hV at eta^m.
 * W or xy may be NULL to leave the term out.
 */
int oracle_advance_ext(void *hm, const double *xy, const double *R_in, const double *W_in, double g_in,
                       double theta_in, double tau, int M, int nonlinear_h, double Abg, double Cv, int nsteps,
                       double *eta_io, double *U_io, double *Umean_out)
{
    omesh *m = (omesh *)hm;
    if (M < 1) return -5;
    const int ne = m->ne, nv = m->nv;
    const real dt = (real)(tau / (double)M);
    const real g = (real)g_in, theta = (real)theta_in;
    real *F = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *U = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *U0 = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *sumU = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *R = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *V0 = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *Vm = (real *)malloc(sizeof(real) * 2 * (size_t)ne);
    real *W = (real *)calloc((size_t)nv, sizeof(real));
    real *eta = (real *)malloc(sizeof(real) * (size_t)nv);
    real *div = (real *)malloc(sizeof(real) * (size_t)nv);
    real *ef = (real *)malloc(sizeof(real) * (size_t)m->ned);
    if (!F || !U || !U0 || !sumU || !R || !V0 || !Vm || !W || !eta || !div || !ef) {
        free(F); free(U); free(U0); free(sumU); free(R); free(V0); free(Vm); free(W); free(eta); free(div); free(ef);
        return -4;
    }
    for (size_t i = 0; i < 2 * (size_t)ne; i++) { U[i] = (real)U_io[i]; R[i] = (real)R_in[i]; }
    for (int v = 0; v < nv; v++) { eta[v] = (real)eta_io[v]; if (W_in) W[v] = (real)W_in[v]; }
    for (int n = 0; n < nsteps; n++) {
        memcpy(U0, U, sizeof(real) * 2 * (size_t)ne);
        memset(sumU, 0, sizeof(real) * 2 * (size_t)ne);
        if (xy) viscosity(m, U, eta, nonlinear_h, (real)Abg, (real)Cv, xy, V0);
        for (int s = 0; s < M; s++) {
            if (xy) viscosity(m, U, eta, nonlinear_h, (real)Abg, (real)Cv, xy, Vm);
            #pragma omp parallel for schedule(static)
            for (int e = 0; e < ne; e++) {
                real gx, gy;
                gradient_e(m, e, eta, &gx, &gy);
                real H = element_depth(m, e, eta, nonlinear_h);
                real a = dt * m->f_e[e] / 2;
                real ux = U[2 * e], uy = U[2 * e + 1];
                real rx = R[2 * e], ry = R[2 * e + 1];
                if (xy) { rx += Vm[2 * e] - V0[2 * e]; ry += Vm[2 * e + 1] - V0[2 * e + 1]; }
                real A11 = 1, A12 = -a, A21 = a, A22 = 1;
                real bx = ux + a * uy + dt * (-g * H * gx + rx);
                real by = -a * ux + uy + dt * (-g * H * gy + ry);
                real det = A11 * A22 - A12 * A21;
                real nx = (bx * A22 - A12 * by) / det;
                real ny = (A11 * by - A21 * bx) / det;
                F[2 * e] = (1 + theta) * nx - theta * ux;
                F[2 * e + 1] = (1 + theta) * ny - theta * uy;
                U[2 * e] = nx;
                U[2 * e + 1] = ny;
                sumU[2 * e] += nx;
                sumU[2 * e + 1] += ny;
            }
            divergence(m, F, ef, div);
            #pragma omp parallel for schedule(static)
            for (int v = 0; v < nv; v++) eta[v] -= dt * (div[v] + W[v]);
        }
        for (int e = 0; e < ne; e++)
            for (int c = 0; c < 2; c++)
                Umean_out[2 * e + c] = (double)(sumU[2 * e + c] / (real)M + theta / (real)M * (U[2 * e + c] - U0[2 * e + c]));
    }
    for (size_t i = 0; i < 2 * (size_t)ne; i++) U_io[i] = (double)U[i];
    for (int v = 0; v < nv; v++) eta_io[v] = (double)eta[v];
    free(F); free(U); free(U0); free(sumU); free(R); free(V0); free(Vm); free(W); free(eta); free(div); free(ef);
    return 0;
}

int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
