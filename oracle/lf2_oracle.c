/*
 * lf2_oracle.c -- TEST INFRASTRUCTURE, not part of the library.
 *
 * A plain, slow, FP64 CPU statement of the leapfrog lattice-field step.  It exists only so
 * that the test-suite, the smoke check and the CPU-baseline leg of the benchmark can check
 * the CUDA path against something obviously correct.  The library never links, loads or
 * calls it, and it shares no code, header or constant with the CUDA sources.
 *
 * It follows the data model of LATfield2 (Daverio, Hindmarsh & Bevis, arXiv:1508.05610):
 *   - Lattice(dim, sizes, h): an n-D cartesian lattice with a halo of h sites in every
 *     dimension (Sec. 3.2, Sec. 3.3.1);
 *   - Field: per-site component lists stored in row-major order, dimension 0 fastest,
 *     halo included (Sec. 3.3, Sec. 3.4);
 *   - updateHalo(): copies the periodic image of the interior into the halo, which is how
 *     the library encodes the torus topology (Sec. 3.3.1);
 *   - Site: a memory index walked by first()/test()/next(); x+i / x-i add or subtract the
 *     "jump" of dimension i, which is 1 in dimension 0 and (N0 + 2h) in dimension 1, and so
 *     on (Sec. 3.4).
 *
 * The physics is not written down in the paper; the paper's field-evolution applications
 * (Sec. 1, Sec. 5) are classical scalar fields.  The oracle uses these readings:
 *   - equation of motion  d2phi_a/dt2 = lap phi_a - dV/dphi_a  with
 *     V = (lambda/4)(sum_b phi_b^2 - eta^2)^2 + (m2/2) sum_a phi_a^2 (real-component form,
 *     one or two components);
 *   - lap is the 7-point lattice Laplacian (1/dx^2) sum_i [phi(x+i) + phi(x-i) - 2 phi(x)];
 *   - staggered leapfrog: pi lives at half steps, pi_{-1/2} = pi_0 - (dt/2) F(phi_0), then
 *     each step  pi_{n+1/2} = pi_{n-1/2} + dt F(phi_n);  phi_{n+1} = phi_n + dt pi_{n+1/2};
 *   - energy at integer step n with the synchronised pi_n = pi_{n-1/2} + (dt/2) F(phi_n),
 *     forward-difference gradient energy (the one whose variation is the 7-point Laplacian)
 *     and volume element dx^3; sums are Neumaier-compensated.
 *
 * Everything is FP64.  The one OpenMP pragma splits the site loops over z-planes for the
 * timed CPU baseline only: each site's arithmetic is the same, so results are bitwise equal
 * for any thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_EINVAL 1
#define ORA_ENOMEM 3

/* ---------------------------------------------------------------- Lattice (Sec. 3.2) */
typedef struct {
    int dim;           /* always 3 here */
    int n[3];          /* interior sizes N0, N1, N2 */
    int h;             /* halo width */
    long pad[3];       /* padded sizes N_i + 2h */
    long jump[3];      /* Site jumps: 1, pad0, pad0*pad1 (Sec. 3.4) */
    long sites_padded; /* pad0*pad1*pad2 */
} ora_lattice;

static int lattice_init(ora_lattice *lat, const int *sizes, int h) {
    if (h < 1) return ORA_EINVAL;
    lat->dim = 3;
    lat->h = h;
    for (int i = 0; i < 3; ++i) {
        if (sizes[i] < 1) return ORA_EINVAL;
        lat->n[i] = sizes[i];
        lat->pad[i] = sizes[i] + 2L * h;
    }
    lat->jump[0] = 1;
    lat->jump[1] = lat->pad[0];
    lat->jump[2] = lat->pad[0] * lat->pad[1];
    lat->sites_padded = lat->pad[0] * lat->pad[1] * lat->pad[2];
    return ORA_OK;
}

/* ------------------------------------------------------------------ Field (Sec. 3.3) */
typedef struct {
    const ora_lattice *lat;
    int comp;
    double *data; /* sites_padded * comp, component list per site */
} ora_field;

static int field_alloc(ora_field *f, const ora_lattice *lat, int comp) {
    f->lat = lat;
    f->comp = comp;
    f->data = (double *)calloc((size_t)lat->sites_padded * (size_t)comp, sizeof(double));
    return f->data ? ORA_OK : ORA_ENOMEM;
}

static void field_free(ora_field *f) {
    free(f->data);
    f->data = NULL;
}

/* ------------------------------------------------------------------- Site (Sec. 3.4) */
typedef struct {
    const ora_lattice *lat;
    long index;   /* memory index of the site, halo included */
    int coord[3]; /* interior coordinate */
} ora_site;

static long site_index_of(const ora_lattice *lat, const int *coord) {
    return (long)(coord[0] + lat->h) * lat->jump[0] + (long)(coord[1] + lat->h) * lat->jump[1] +
           (long)(coord[2] + lat->h) * lat->jump[2];
}

static void site_first(ora_site *x, const ora_lattice *lat) {
    x->lat = lat;
    x->coord[0] = x->coord[1] = x->coord[2] = 0;
    x->index = site_index_of(lat, x->coord);
}

static int site_test(const ora_site *x) { return x->coord[2] < x->lat->n[2]; }

/* Walks the interior in memory order: dimension 0 fastest, then 1, then 2. */
static void site_next(ora_site *x) {
    const ora_lattice *lat = x->lat;
    for (int d = 0; d < 3; ++d) {
        x->coord[d] += 1;
        if (x->coord[d] < lat->n[d] || d == 2) break;
        x->coord[d] = 0;
    }
    if (x->coord[2] < lat->n[2]) x->index = site_index_of(lat, x->coord);
}

/* x+i and x-i: the neighbour's memory index (Sec. 3.4). */
static long site_up(const ora_site *x, int i) { return x->index + x->lat->jump[i]; }
static long site_dn(const ora_site *x, int i) { return x->index - x->lat->jump[i]; }

/* ------------------------------------------------------ updateHalo (Sec. 3.3.1) */
/* For each dimension d in turn, every padded site whose d-coordinate lies in the halo takes
 * the value of its periodic image in the interior.  Doing the dimensions one after another
 * over the full padded extent of the other dimensions fills faces, edges and corners. */
static void update_halo(ora_field *f) {
    const ora_lattice *lat = f->lat;
    const int h = lat->h, c = f->comp;
    long p[3];
    for (int d = 0; d < 3; ++d) {
        const long nd = lat->n[d];
        for (p[2] = 0; p[2] < lat->pad[2]; ++p[2])
            for (p[1] = 0; p[1] < lat->pad[1]; ++p[1])
                for (p[0] = 0; p[0] < lat->pad[0]; ++p[0]) {
                    long src_d;
                    if (p[d] < h)
                        src_d = p[d] + nd;
                    else if (p[d] >= nd + h)
                        src_d = p[d] - nd;
                    else
                        continue;
                    const long dst = p[0] * lat->jump[0] + p[1] * lat->jump[1] + p[2] * lat->jump[2];
                    const long src = dst + (src_d - p[d]) * lat->jump[d];
                    for (int a = 0; a < c; ++a) f->data[dst * c + a] = f->data[src * c + a];
                }
    }
}

/* ------------------------------------------------------------- model parameters */
typedef struct {
    double dx, dt, lambda, eta, m2;
} ora_params;

static ora_params params_from(const double *p) {
    ora_params q;
    q.dx = p[0];
    q.dt = p[1];
    q.lambda = p[2];
    q.eta = p[3];
    q.m2 = p[4];
    return q;
}

/* Force on component a at site x, halo already up to date:
 *   F_a = (1/dx^2) [ sum over the 6 neighbours of phi_a ] - 6 phi_a / dx^2
 *         - lambda phi_a (sum_b phi_b^2 - eta^2) - m2 phi_a                              */
static double force_at(const ora_field *phi, const ora_site *x, int a, const ora_params *q) {
    const int c = phi->comp;
    const double *d = phi->data;
    double nb = 0.0;
    for (int i = 0; i < 3; ++i) {
        nb += d[site_dn(x, i) * c + a];
        nb += d[site_up(x, i) * c + a];
    }
    const double here = d[x->index * c + a];
    double s2 = 0.0;
    for (int b = 0; b < c; ++b) s2 += d[x->index * c + b] * d[x->index * c + b];
    const double lap = nb / (q->dx * q->dx) - 6.0 * here / (q->dx * q->dx);
    return lap - q->lambda * here * (s2 - q->eta * q->eta) - q->m2 * here;
}

/* ------------------------------------------------------------- Neumaier summation */
typedef struct {
    double s, c;
} ora_sum;

static void sum_add(ora_sum *acc, double v) {
    const double t = acc->s + v;
    if (fabs(acc->s) >= fabs(v))
        acc->c += (acc->s - t) + v;
    else
        acc->c += (v - t) + acc->s;
    acc->s = t;
}

static double sum_value(const ora_sum *acc) { return acc->s + acc->c; }

/* --------------------------------------------------------- host array <-> Field */
/* The caller's arrays hold only the interior, row-major with dimension 0 fastest and the
 * components of a site next to each other: the paper's binary file layout (Sec. 3.5). */
static void field_load(ora_field *f, const double *host) {
    ora_site x;
    long k = 0;
    for (site_first(&x, f->lat); site_test(&x); site_next(&x))
        for (int a = 0; a < f->comp; ++a) f->data[x.index * f->comp + a] = host[k++];
}

static void field_store(const ora_field *f, double *host) {
    ora_site x;
    long k = 0;
    for (site_first(&x, f->lat); site_test(&x); site_next(&x))
        for (int a = 0; a < f->comp; ++a) host[k++] = f->data[x.index * f->comp + a];
}

/* Points a Site at interior coordinate (x, y, z); used to split the Site loop into
 * independent z-planes for the OpenMP-timed variant. */
static void site_set(ora_site *s, const ora_lattice *lat, int x, int y, int z) {
    s->lat = lat;
    s->coord[0] = x;
    s->coord[1] = y;
    s->coord[2] = z;
    s->index = site_index_of(lat, s->coord);
}

/* pi <- pi + scale * F(phi), halo of phi up to date. */
static void kick(ora_field *pi, const ora_field *phi, double scale, const ora_params *q,
                 int nthreads) {
    const ora_lattice *lat = phi->lat;
    const int c = phi->comp;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int z = 0; z < lat->n[2]; ++z)
        for (int y = 0; y < lat->n[1]; ++y)
            for (int xx = 0; xx < lat->n[0]; ++xx) {
                ora_site x;
                site_set(&x, lat, xx, y, z);
                double F[8];
                for (int a = 0; a < c; ++a) F[a] = force_at(phi, &x, a, q);
                for (int a = 0; a < c; ++a) pi->data[x.index * c + a] += scale * F[a];
            }
}

/* phi_new <- phi + dt * pi on the interior. */
static void drift(ora_field *phi_new, const ora_field *phi, const ora_field *pi, double dt,
                  int nthreads) {
    const ora_lattice *lat = phi->lat;
    const int c = phi->comp;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int z = 0; z < lat->n[2]; ++z)
        for (int y = 0; y < lat->n[1]; ++y)
            for (int xx = 0; xx < lat->n[0]; ++xx) {
                ora_site x;
                site_set(&x, lat, xx, y, z);
                for (int a = 0; a < c; ++a)
                    phi_new->data[x.index * c + a] =
                        phi->data[x.index * c + a] + dt * pi->data[x.index * c + a];
            }
}

static int check_shape(int nx, int ny, int nz, int ncomp) {
    if (nx < 1 || ny < 1 || nz < 1) return ORA_EINVAL;
    if (ncomp < 1 || ncomp > 8) return ORA_EINVAL;
    return ORA_OK;
}

/* ==================================================================== exported API */

/* Fills the halo of a padded array (sizes + 2 per dimension, halo 1) in place. */
int ora_update_halo(int nx, int ny, int nz, int ncomp, double *padded) {
    const int sizes[3] = {nx, ny, nz};
    ora_lattice lat;
    if (check_shape(nx, ny, nz, ncomp) || lattice_init(&lat, sizes, 1)) return ORA_EINVAL;
    ora_field f = {&lat, ncomp, padded};
    update_halo(&f);
    return ORA_OK;
}

/* F(phi) at every interior site; phi and F are interior arrays. */
int ora_force(int nx, int ny, int nz, int ncomp, const double *params, const double *phi_host,
              double *force_out) {
    const int sizes[3] = {nx, ny, nz};
    ora_lattice lat;
    if (check_shape(nx, ny, nz, ncomp) || lattice_init(&lat, sizes, 1)) return ORA_EINVAL;
    const ora_params q = params_from(params);
    ora_field phi;
    if (field_alloc(&phi, &lat, ncomp)) return ORA_ENOMEM;
    field_load(&phi, phi_host);
    update_halo(&phi);
    ora_site x;
    long k = 0;
    for (site_first(&x, &lat); site_test(&x); site_next(&x))
        for (int a = 0; a < ncomp; ++a) force_out[k++] = force_at(&phi, &x, a, &q);
    field_free(&phi);
    return ORA_OK;
}

/* Leapfrog evolution in place on interior arrays phi (phi_n) and pi (pi_{n-1/2}).
 * half_kick != 0 first turns pi_0 into pi_{-1/2} = pi_0 - (dt/2) F(phi_0).
 * Then nsteps steps of: updateHalo(phi); pi += dt F(phi); phi_new = phi + dt pi; swap. */
int ora_evolve(int nx, int ny, int nz, int ncomp, const double *params, double *phi_host,
               double *pi_host, int nsteps, int half_kick, int nthreads) {
    const int sizes[3] = {nx, ny, nz};
    ora_lattice lat;
    if (check_shape(nx, ny, nz, ncomp) || lattice_init(&lat, sizes, 1) || nsteps < 0) return ORA_EINVAL;
    const ora_params q = params_from(params);
    ora_field phi, phi_new, pi;
    if (field_alloc(&phi, &lat, ncomp)) return ORA_ENOMEM;
    if (field_alloc(&phi_new, &lat, ncomp)) {
        field_free(&phi);
        return ORA_ENOMEM;
    }
    if (field_alloc(&pi, &lat, ncomp)) {
        field_free(&phi);
        field_free(&phi_new);
        return ORA_ENOMEM;
    }
    field_load(&phi, phi_host);
    field_load(&pi, pi_host);
    if (half_kick) {
        update_halo(&phi);
        kick(&pi, &phi, -0.5 * q.dt, &q, nthreads);
    }
    for (int n = 0; n < nsteps; ++n) {
        update_halo(&phi);
        kick(&pi, &phi, q.dt, &q, nthreads);
        drift(&phi_new, &phi, &pi, q.dt, nthreads);
        ora_field t = phi;
        phi = phi_new;
        phi_new = t;
    }
    field_store(&phi, phi_host);
    field_store(&pi, pi_host);
    field_free(&phi);
    field_free(&phi_new);
    field_free(&pi);
    return ORA_OK;
}

/* First-order symmetric difference along dimension i, the paper's example of Site use
 * (Sec. 3.4): d_a(x) = (phi_a(x+i) - phi_a(x-i)) / (2 dx), for every component, into a second
 * field -- the "field operation" the paper benchmarks (Sec. 4.2). */
int ora_derivative(int nx, int ny, int nz, int ncomp, int dim, double dx, const double *phi_host,
                   double *out_host) {
    const int sizes[3] = {nx, ny, nz};
    ora_lattice lat;
    if (check_shape(nx, ny, nz, ncomp) || lattice_init(&lat, sizes, 1) || dim < 0 || dim > 2 || !(dx > 0.0))
        return ORA_EINVAL;
    ora_field phi, out;
    if (field_alloc(&phi, &lat, ncomp)) return ORA_ENOMEM;
    if (field_alloc(&out, &lat, ncomp)) {
        field_free(&phi);
        return ORA_ENOMEM;
    }
    field_load(&phi, phi_host);
    update_halo(&phi);
    ora_site x;
    for (site_first(&x, &lat); site_test(&x); site_next(&x))
        for (int a = 0; a < ncomp; ++a)
            out.data[x.index * ncomp + a] =
                (phi.data[site_up(&x, dim) * ncomp + a] - phi.data[site_dn(&x, dim) * ncomp + a]) / (2.0 * dx);
    field_store(&out, out_host);
    field_free(&phi);
    field_free(&out);
    return ORA_OK;
}

/* Energy and checksums at integer step n from phi_n and pi_{n-1/2}.
 * out[0..3] = kinetic, gradient, potential, total (each with the dx^3 volume element);
 * out[4..4+ncomp) = sum_x phi_a;  out[4+ncomp..4+2 ncomp) = sum_x phi_a^2.              */
int ora_energy(int nx, int ny, int nz, int ncomp, const double *params, const double *phi_host,
               const double *pi_host, double *out) {
    const int sizes[3] = {nx, ny, nz};
    ora_lattice lat;
    if (check_shape(nx, ny, nz, ncomp) || lattice_init(&lat, sizes, 1)) return ORA_EINVAL;
    const ora_params q = params_from(params);
    ora_field phi, pi;
    if (field_alloc(&phi, &lat, ncomp)) return ORA_ENOMEM;
    if (field_alloc(&pi, &lat, ncomp)) {
        field_free(&phi);
        return ORA_ENOMEM;
    }
    field_load(&phi, phi_host);
    field_load(&pi, pi_host);
    update_halo(&phi);

    ora_sum kin = {0, 0}, grad = {0, 0}, pot = {0, 0};
    ora_sum sum[8], sumsq[8];
    memset(sum, 0, sizeof sum);
    memset(sumsq, 0, sizeof sumsq);
    const double dx2 = q.dx * q.dx;
    ora_site x;
    for (site_first(&x, &lat); site_test(&x); site_next(&x)) {
        double s2 = 0.0;
        for (int a = 0; a < ncomp; ++a) {
            const double v = phi.data[x.index * ncomp + a];
            /* synchronised momentum pi_n = pi_{n-1/2} + (dt/2) F(phi_n) */
            const double pin = pi.data[x.index * ncomp + a] + 0.5 * q.dt * force_at(&phi, &x, a, &q);
            sum_add(&kin, 0.5 * pin * pin);
            for (int i = 0; i < 3; ++i) {
                const double dphi = phi.data[site_up(&x, i) * ncomp + a] - v;
                sum_add(&grad, 0.5 * dphi * dphi / dx2);
            }
            s2 += v * v;
            sum_add(&sum[a], v);
            sum_add(&sumsq[a], v * v);
        }
        const double w = s2 - q.eta * q.eta;
        sum_add(&pot, 0.25 * q.lambda * w * w + 0.5 * q.m2 * s2);
    }
    const double vol = q.dx * q.dx * q.dx;
    out[0] = vol * sum_value(&kin);
    out[1] = vol * sum_value(&grad);
    out[2] = vol * sum_value(&pot);
    out[3] = out[0] + out[1] + out[2];
    for (int a = 0; a < ncomp; ++a) {
        out[4 + a] = sum_value(&sum[a]);
        out[4 + ncomp + a] = sum_value(&sumsq[a]);
    }
    field_free(&phi);
    field_free(&pi);
    return ORA_OK;
}
