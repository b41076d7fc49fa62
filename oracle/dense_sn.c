/* Dense full-grid FP64 multigroup S_N step: the oracle's traditional solver
 * (TEST INFRASTRUCTURE: only tests, smoke() and bench's cpu_baseline/reference arm run it).
 *
 * One step = forward-Euler upwind transport (Sec. 2.1 first paragraph; Appendix A,
 * 'Value of n': T_x I_i = (dt/dx)(F_{i+1/2} - F_{i-1/2}) with upwind F), applied with a
 * minus sign as conservation requires, followed by the backward-Euler operator-split
 * absorption/emission/scattering update of Eq. (discRTsource) at fixed material
 * temperature (epsilon^{m+1} = epsilon):
 *
 *   I*_i   = I_i - sum_axes lam_a * ( n_a >= 0 ? n_a (I_i - I_{i-1}) : n_a (I_{i+1} - I_i) )
 *   J*     = (1/4pi) sum_angles dOmega I*
 *   J^{m+1}= (J* + a eps) / (1 + a)                           a = c dt rho kappa_a
 *   I^{m+1}= (I* + a eps + s J^{m+1}) / (1 + a + s)           s = c dt rho kappa_s
 *
 * Ghost cells hold the face's isotropic inflow spectrum, or 0 for vacuum.
 *
 * flux = 1 replaces the upwind flux by the Rusanov flux of Appendix A ('Value of n'):
 * F_{i+1/2} = n (I_i + I_{i+1}) / 2 - alpha (I_{i+1} - I_i) / 2 with alpha = 1 (the largest
 * speed, c |n| <= c), i.e. T I_i = lam [ n (I_{i+1} - I_{i-1}) / 2 - (I_{i+1} - 2 I_i + I_{i-1}) / 2 ],
 * read with vacuum ghost cells (0) on every face.  alpha_local = 1 takes alpha = |n| per direction
 * instead, which is the upwind flux again (a consistency check of the two schemes).  flux = 2 is
 * the Rusanov flux with wavespeed S+ = alpha = 0, the pure central difference of Sec. 4.3.
 * Layout: I[k * nang + q], merged row k = g + G*(ix + nx*(iy + ny*iz)), angle q.
 */
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdlib.h>
#include <string.h>

typedef struct {
    int ndim, nx, ny, nz, G, nang;
    const double *dir[3];   /* direction cosine per angle for axes x, y, z */
    const double *domega;   /* solid-angle weight per angle (sum 4 pi) */
    double lam[3];          /* c dt / dx_a */
    const double *acoef;    /* per row: c dt rho kappa_a */
    const double *scoef;    /* per row: c dt rho kappa_s */
    const double *eps;      /* per row: emission epsilon_f(T) */
    const double *inflow[6];/* per face (x-,x+,y-,y+,z-,z+): G-spectrum or NULL (vacuum) */
    int flux;               /* 0 upwind, 1 Rusanov, 2 central (vacuum ghost cells) */
    int alpha_local;        /* Rusanov with alpha = |n| (reduces to upwind) */
} dense_params;

static double ghost(const dense_params *p, int face, int g) {
    return p->inflow[face] ? p->inflow[face][g] : 0.0;
}

/* I -> Iout (one full step).  If Istar is not NULL it receives the post-transport field. */
int dense_step(const dense_params *p, const double *I, double *Iout, double *Istar) {
    const long nrow = (long)p->nx * p->ny * p->nz * p->G;
    const int nang = p->nang;
    const long stride[3] = {(long)p->G, (long)p->G * p->nx, (long)p->G * p->nx * p->ny};
    const int extent[3] = {p->nx, p->ny, p->nz};
    int err = 0;
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * (size_t)nang);
        if (!buf) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(static)
        for (long k = 0; k < nrow; ++k) {
            if (!buf) continue;
            const int g = (int)(k % p->G);
            long cell = k / p->G;
            int idx[3];
            idx[0] = (int)(cell % p->nx);
            idx[1] = (int)((cell / p->nx) % p->ny);
            idx[2] = (int)(cell / ((long)p->nx * p->ny));
            const double *Ik = I + k * nang;
            for (int q = 0; q < nang; ++q) {
                double v = Ik[q];
                double acc = 0.0;
                for (int ax = 0; ax < p->ndim; ++ax) {
                    double n = p->dir[ax][q];
                    if (p->flux == 1 || p->flux == 2) {
                        const double lo = (idx[ax] > 0) ? I[(k - stride[ax]) * nang + q] : 0.0;
                        const double hi = (idx[ax] < extent[ax] - 1) ? I[(k + stride[ax]) * nang + q] : 0.0;
                        const double alpha = (p->flux == 2) ? 0.0 : (p->alpha_local ? fabs(n) : 1.0);
                        acc += p->lam[ax] * (0.5 * n * (hi - lo) - 0.5 * alpha * (hi - 2.0 * v + lo));
                        continue;
                    }
                    if (n >= 0.0) {
                        double up = (idx[ax] > 0) ? I[(k - stride[ax]) * nang + q] : ghost(p, 2 * ax, g);
                        acc += p->lam[ax] * n * (v - up);
                    } else {
                        double dn = (idx[ax] < extent[ax] - 1) ? I[(k + stride[ax]) * nang + q]
                                                               : ghost(p, 2 * ax + 1, g);
                        acc += p->lam[ax] * n * (dn - v);
                    }
                }
                buf[q] = v - acc;
            }
            double js = 0.0;
            for (int q = 0; q < nang; ++q) js += p->domega[q] * buf[q];
            js /= 4.0 * M_PI;
            const double a = p->acoef[k], s = p->scoef[k], e = p->eps[k];
            const double jn = (js + a * e) / (1.0 + a);
            const double rhs = a * e + s * jn;
            const double den = 1.0 + a + s;
            for (int q = 0; q < nang; ++q) {
                Iout[k * nang + q] = (buf[q] + rhs) / den;
                if (Istar) Istar[k * nang + q] = buf[q];
            }
        }
        free(buf);
    }
    return err;
}

int dense_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
