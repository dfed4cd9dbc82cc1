/*
 * Plain FP64 CPU oracle for the heat-diffusion hot path of
 * "Distributed Parallelization of xPU Stencil Computations in Julia"
 * (Omlin, Raess, Utkin; JuliaCon proceedings, arXiv 2211.15716).
 *
 * TEST INFRASTRUCTURE. This file is the slow, obviously correct statement of
 * what the GPU library computes. Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it. It shares no code, header or
 * constant with the CUDA library, and the CUDA library never loads it.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp].
 * -ffp-contract=off keeps every + - * / a separately rounded IEEE operation,
 * so the arithmetic below is exactly the expression printed in Fig. 1.
 * The OpenMP pragmas only split independent cells between threads; results
 * are identical with and without them.
 *
 * Layout of every field: x fastest, then y, then z (Julia column-major order,
 * Fig. 1), linear index p = ix + nx*(iy + ny*iz), 0-based.
 * A field on a grid of nsub subdomains is one buffer [nsub][nz][ny][nx].
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(ix, iy, iz) ((size_t)(ix) + (size_t)nx * ((size_t)(iy) + (size_t)ny * (size_t)(iz)))

/* One inner cell of Fig. 1's step! kernel:
 *   T2 = T + dt*(lam*Ci*(d2x/dx^2 + d2y/dy^2 + d2z/dz^2))
 * with the second difference along x read as the difference of the two
 * one-sided differences, (T[x+1]-T[x]) - (T[x]-T[x-1]) (same for y, z), and
 * dx^2 evaluated as dx*dx. Evaluated left to right as printed. */
static double step_cell(const double *T, const double *Ci, size_t p, size_t sx,
                        size_t sy, size_t sz, double lam, double dt, double dx,
                        double dy, double dz) {
  double d2x = (T[p + sx] - T[p]) - (T[p] - T[p - sx]);
  double d2y = (T[p + sy] - T[p]) - (T[p] - T[p - sy]);
  double d2z = (T[p + sz] - T[p]) - (T[p] - T[p - sz]);
  double lap = ((d2x / (dx * dx)) + (d2y / (dy * dy))) + (d2z / (dz * dz));
  return T[p] + dt * ((lam * Ci[p]) * lap);
}

/* Laplacian term of step_cell alone (used by the adjoint's Ci gradient). */
static double lap_cell(const double *T, size_t p, size_t sx, size_t sy,
                       size_t sz, double dx, double dy, double dz) {
  double d2x = (T[p + sx] - T[p]) - (T[p] - T[p - sx]);
  double d2y = (T[p + sy] - T[p]) - (T[p] - T[p - sy]);
  double d2z = (T[p + sz] - T[p]) - (T[p] - T[p - sz]);
  return ((d2x / (dx * dx)) + (d2y / (dy * dy))) + (d2z / (dz * dz));
}

/* A dimension of size 1 is absent (a 2-D or 1-D grid): its only index counts
 * as inner and its neighbour stride is 0, so its second difference is exactly
 * 0 (with an infinite spacing its term d2/(dd*dd) is 0 as well). */
#define LO(n) ((n) > 1 ? 1L : 0L)
#define HI(n) ((n) > 1 ? (n) - 1 : 1L)

/* Fig. 1 step! on one local array: every inner point (index 1..n-2 in each
 * dimension, 0-based) of T2 is written; points on the array boundary are not
 * touched (they keep whatever T2 holds, which is how Fig. 1's T2 = copy(T)
 * yields fixed boundary values). */
void oracle_step(long nx, long ny, long nz, double *T2, const double *T,
                 const double *Ci, double lam, double dt, double dx, double dy,
                 double dz) {
  const size_t sx = nx > 1 ? 1 : 0, sy = ny > 1 ? (size_t)nx : 0,
               sz = nz > 1 ? (size_t)nx * (size_t)ny : 0;
#pragma omp parallel for schedule(static)
  for (long iz = LO(nz); iz < HI(nz); ++iz)
    for (long iy = LO(ny); iy < HI(ny); ++iy)
      for (long ix = LO(nx); ix < HI(nx); ++ix) {
        size_t p = AT(ix, iy, iz);
        T2[p] = step_cell(T, Ci, p, sx, sy, sz, lam, dt, dx, dy, dz);
      }
}

/* The same update restricted to inner points inside a box, either the
 * boundary set (select = 1) or the inner block (select = 0) of the
 * boundary/inner split used by hide_communication (Fig. 1, the
 * @hide_communication (16, 2, 2) block; Sec. Approach).
 * Boundary set: inner points whose 1-based index i satisfies i <= w or
 * i >= n - w + 1 in at least one dimension, w the width of that dimension.
 * Inner block: all other inner points. */
static int in_boundary_set(long i, long n, long w) {
  /* 0-based i; 1-based i+1 <= w  or  i+1 >= n-w+1; an absent dimension
   * (n = 1) has no boundary slab */
  return n > 1 && ((i + 1 <= w) || (i + 1 >= n - w + 1));
}

void oracle_step_part(long nx, long ny, long nz, double *T2, const double *T,
                      const double *Ci, double lam, double dt, double dx,
                      double dy, double dz, long bx, long by, long bz,
                      int select) {
  const size_t sx = nx > 1 ? 1 : 0, sy = ny > 1 ? (size_t)nx : 0,
               sz = nz > 1 ? (size_t)nx * (size_t)ny : 0;
#pragma omp parallel for schedule(static)
  for (long iz = LO(nz); iz < HI(nz); ++iz)
    for (long iy = LO(ny); iy < HI(ny); ++iy)
      for (long ix = LO(nx); ix < HI(nx); ++ix) {
        int b = in_boundary_set(ix, nx, bx) || in_boundary_set(iy, ny, by) ||
                in_boundary_set(iz, nz, bz);
        if (b != select) continue;
        size_t p = AT(ix, iy, iz);
        T2[p] = step_cell(T, Ci, p, sx, sy, sz, lam, dt, dx, dy, dz);
      }
}

/* Halo update of one field on a grid of nsub subdomains (update_halo!,
 * Sec. Approach; Fig. 1 update_halo!(T2)). Halo width 1, overlap o[d] >= 2.
 * Dimensions are processed in the order x, y, z. Within dimension d, every
 * subdomain S receives:
 *   - its first plane (index 0) from plane n-o of its left neighbour,
 *   - its last plane (index n-1) from plane o-1 of its right neighbour,
 * where left_nb[3*S+d] / right_nb[3*S+d] is the neighbour's subdomain number,
 * or -1 for none (a physical boundary). Whole planes are copied, including the
 * points that lie in other dimensions' halos, so the x, y, z order decides the
 * values of edges and corners. The copy is a byte copy of elem_size bytes per
 * point, so it serves every element type. A dimension whose overlap is below
 * 2 exchanges nothing (a staggered field's overlap o + (n_f - n) can be 1:
 * the neighbours then share one plane and have no halo plane to fill). */
void oracle_update_halo(int nsub, const int *left_nb, const int *right_nb,
                        long nx, long ny, long nz, const long *overlap,
                        void *field, long elem_size) {
  const long n[3] = {nx, ny, nz};
  const size_t nloc = (size_t)nx * (size_t)ny * (size_t)nz;
  unsigned char *base = (unsigned char *)field;
  const size_t es = (size_t)elem_size;
  for (int d = 0; d < 3; ++d) {
    const long o = overlap[d];
    if (o < 2 || n[d] < 2) continue; /* staggered overlap 1, or an absent dimension */
    for (int s = 0; s < nsub; ++s) {
      for (int side = 0; side < 2; ++side) {
        int nb = side == 0 ? left_nb[3 * s + d] : right_nb[3 * s + d];
        if (nb < 0) continue;
        long dst_plane = side == 0 ? 0 : n[d] - 1;
        long src_plane = side == 0 ? n[d] - o : o - 1;
        unsigned char *dst = base + (size_t)s * nloc * es;
        const unsigned char *src = base + (size_t)nb * nloc * es;
        /* every point of the plane: the two other dimensions a, b, all indices */
        const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;
        for (long ib = 0; ib < n[db]; ++ib)
          for (long ia = 0; ia < n[da]; ++ia) {
            long c[3], cs[3];
            c[d] = dst_plane;
            cs[d] = src_plane;
            c[da] = cs[da] = ia;
            c[db] = cs[db] = ib;
            memcpy(dst + AT(c[0], c[1], c[2]) * es, src + AT(cs[0], cs[1], cs[2]) * es, es);
          }
      }
    }
  }
}

/* The adjoint (transpose) of the halo update above on an FP64 field: the
 * update is a product of plane copies, dimensions x, then y, then z, and
 * each copy field[dst] = field[src] is the linear map that replaces the
 * dst entry by the src entry. Its transpose adds the dst entry into the src
 * entry and sets the dst entry to 0. The transpose of the product takes the
 * dimensions in the reverse order: z, then y, then x. Within one dimension
 * the copies' dst planes (0 and n-1) and src planes (o-1 and n-o) are
 * distinct, so their order does not matter. */
void oracle_update_halo_adjoint(int nsub, const int *left_nb, const int *right_nb,
                                long nx, long ny, long nz, const long *overlap,
                                double *lam) {
  const long n[3] = {nx, ny, nz};
  const size_t nloc = (size_t)nx * (size_t)ny * (size_t)nz;
  for (int d = 2; d >= 0; --d) {
    const long o = overlap[d];
    if (o < 2 || n[d] < 2) continue;
    for (int s = 0; s < nsub; ++s) {
      for (int side = 0; side < 2; ++side) {
        int nb = side == 0 ? left_nb[3 * s + d] : right_nb[3 * s + d];
        if (nb < 0) continue;
        long dst_plane = side == 0 ? 0 : n[d] - 1;
        long src_plane = side == 0 ? n[d] - o : o - 1;
        double *dst = lam + (size_t)s * nloc;
        double *src = lam + (size_t)nb * nloc;
        const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;
        for (long ib = 0; ib < n[db]; ++ib)
          for (long ia = 0; ia < n[da]; ++ia) {
            long c[3], cs[3];
            c[d] = dst_plane;
            cs[d] = src_plane;
            c[da] = cs[da] = ia;
            c[db] = cs[db] = ib;
            src[AT(cs[0], cs[1], cs[2])] += dst[AT(c[0], c[1], c[2])];
            dst[AT(c[0], c[1], c[2])] = 0.0;
          }
      }
    }
  }
}

/* One backward step of the discrete adjoint of Fig. 1's step! (the transposed
 * stencil run backward in time; the gradient form of the step).
 * Forward: T_{n+1}[p] = T_n[p] + dt*lam*Ci[p]*(L T_n)[p] on inner p, identity
 * elsewhere, with L the 7-point operator of step_cell.
 * Given lam_in = dJ/dT_{n+1}, writes lam_out = dJ/dT_n:
 *   v[p] = Ci[p]*lam_in[p] on inner p, 0 elsewhere,
 *   lam_out[q] = lam_in[q] + dt*lam*sum_d (v[q+e_d] + v[q-e_d] - 2 v[q]) / dd^2,
 * neighbours outside the array counting as 0; and accumulates
 *   gCi[p] += dt*lam*lam_in[p]*(L T_n)[p] on inner p. */
void oracle_adjoint_step(long nx, long ny, long nz, double *lam_out,
                         const double *lam_in, const double *Tn,
                         const double *Ci, double *gCi, double lam, double dt,
                         double dx, double dy, double dz) {
  const size_t sx = 1, sy = (size_t)nx, sz = (size_t)nx * (size_t)ny;
  const double k = dt * lam;
#pragma omp parallel for schedule(static)
  for (long iz = 0; iz < nz; ++iz)
    for (long iy = 0; iy < ny; ++iy)
      for (long ix = 0; ix < nx; ++ix) {
        const long c[3] = {ix, iy, iz};
        const size_t st[3] = {sx, sy, sz};
        const double w[3] = {1.0 / (dx * dx), 1.0 / (dy * dy), 1.0 / (dz * dz)};
        size_t q = AT(ix, iy, iz);
        double acc = 0.0;
        for (int d = 0; d < 3; ++d) {
          double vp = 0.0, vm = 0.0, vq = 0.0;
          long cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
          cp[d] += 1;
          cm[d] -= 1;
          /* v is nonzero only on inner points */
          int q_in = ix > 0 && ix < nx - 1 && iy > 0 && iy < ny - 1 && iz > 0 && iz < nz - 1;
          int p_in = cp[0] > 0 && cp[0] < nx - 1 && cp[1] > 0 && cp[1] < ny - 1 && cp[2] > 0 && cp[2] < nz - 1;
          int m_in = cm[0] > 0 && cm[0] < nx - 1 && cm[1] > 0 && cm[1] < ny - 1 && cm[2] > 0 && cm[2] < nz - 1;
          if (p_in) vp = Ci[q + st[d]] * lam_in[q + st[d]];
          if (m_in) vm = Ci[q - st[d]] * lam_in[q - st[d]];
          if (q_in) vq = Ci[q] * lam_in[q];
          acc += (vp + vm - 2.0 * vq) * w[d];
        }
        lam_out[q] = lam_in[q] + k * acc;
        if (ix > 0 && ix < nx - 1 && iy > 0 && iy < ny - 1 && iz > 0 && iz < nz - 1)
          gCi[q] += k * lam_in[q] * lap_cell(Tn, q, sx, sy, sz, dx, dy, dz);
      }
}

/* Number of OpenMP threads the loops above use (1 without OpenMP). */
/* One leapfrog step of linear acoustics on a staggered grid: the multi-field
 * staggered stencil that exercises update_halo! on fields of different sizes
 * (the paper's grids are regular staggered grids, Sec. Approach; it prints no
 * such solver, so the scheme is the textbook one, stated here).
 * P is a cell field [nz][ny][nx]; the face fields are Vx [nz][ny][nx+1],
 * Vy [nz][ny+1][nx], Vz [nz+1][ny][nx], face index i lying between cells i-1
 * and i. With rho (density) and K (bulk modulus):
 *   1. Vx[k][j][i] -= dt/rho*(P[k][j][i] - P[k][j][i-1])/dx for faces
 *      i = 1..nx-1 and all j, k (likewise Vy over j = 1..ny-1, Vz over
 *      k = 1..nz-1): the outermost faces (walls) are never written;
 *   2. P[k][j][i] -= dt*K*((Vx[k][j][i+1] - Vx[k][j][i])/dx
 *                         + (Vy[k][j+1][i] - Vy[k][j][i])/dy
 *                         + (Vz[k+1][j][i] - Vz[k][j][i])/dz) on every cell,
 * with the new velocities. Each expression is evaluated left to right. */
void oracle_acoustic_step(long nx, long ny, long nz, double *P, double *Vx, double *Vy,
                          double *Vz, double rho, double K, double dt, double dx, double dy,
                          double dz) {
#define PI(i, j, k) ((size_t)(i) + (size_t)nx * ((size_t)(j) + (size_t)ny * (size_t)(k)))
#define VXI(i, j, k) ((size_t)(i) + (size_t)(nx + 1) * ((size_t)(j) + (size_t)ny * (size_t)(k)))
#define VYI(i, j, k) ((size_t)(i) + (size_t)nx * ((size_t)(j) + (size_t)(ny + 1) * (size_t)(k)))
#define VZI(i, j, k) ((size_t)(i) + (size_t)nx * ((size_t)(j) + (size_t)ny * (size_t)(k)))
  long i, j, k;
#pragma omp parallel for private(i, j)
  for (k = 0; k < nz; ++k)
    for (j = 0; j < ny; ++j)
      for (i = 1; i < nx; ++i)
        Vx[VXI(i, j, k)] = Vx[VXI(i, j, k)] - dt / rho * (P[PI(i, j, k)] - P[PI(i - 1, j, k)]) / dx;
#pragma omp parallel for private(i, j)
  for (k = 0; k < nz; ++k)
    for (j = 1; j < ny; ++j)
      for (i = 0; i < nx; ++i)
        Vy[VYI(i, j, k)] = Vy[VYI(i, j, k)] - dt / rho * (P[PI(i, j, k)] - P[PI(i, j - 1, k)]) / dy;
#pragma omp parallel for private(i, j)
  for (k = 1; k < nz; ++k)
    for (j = 0; j < ny; ++j)
      for (i = 0; i < nx; ++i)
        Vz[VZI(i, j, k)] = Vz[VZI(i, j, k)] - dt / rho * (P[PI(i, j, k)] - P[PI(i, j, k - 1)]) / dz;
#pragma omp parallel for private(i, j)
  for (k = 0; k < nz; ++k)
    for (j = 0; j < ny; ++j)
      for (i = 0; i < nx; ++i)
        P[PI(i, j, k)] = P[PI(i, j, k)] -
                         dt * K *
                             ((Vx[VXI(i + 1, j, k)] - Vx[VXI(i, j, k)]) / dx +
                              (Vy[VYI(i, j + 1, k)] - Vy[VYI(i, j, k)]) / dy +
                              (Vz[VZI(i, j, k + 1)] - Vz[VZI(i, j, k)]) / dz);
#undef PI
#undef VXI
#undef VYI
#undef VZI
}

/* Half steps of a Gross-Pitaevskii solver on one local array (a complex
 * field psi = u + i v on the grid; the paper names a quantum-fluid solver of
 * the nonlinear Gross-Pitaevskii equation as an application of the approach
 * and prints no equations, so they are stated here):
 *   i dpsi/dt = -1/2 lap(psi) + V psi + g |psi|^2 psi,
 * i.e. du/dt = H v, dv/dt = -H u with H w = -1/2 lap(w) + (V + g (u^2 + v^2)) w.
 * Staggered in time (u at whole steps, v at half steps):
 *   which = 0:  u += dt * H(v)   with u^2 + v^2 from the current u and v,
 *   which = 1:  v -= dt * H(u)   with the new u,
 * on inner points only (psi fixed on the array boundary), lap the 7-point
 * operator of step_cell. Each expression is evaluated left to right:
 *   lap = ((d2x/(dx*dx) + d2y/(dy*dy)) + d2z/(dz*dz)),
 *   h   = -0.5*lap + (V[p] + g*(u[p]*u[p] + v[p]*v[p]))*w[p],
 *   out = out + dt*h  (which 0, out = u, w = v)  or  out - dt*h  (which 1,
 *   out = v, w = u). */
void oracle_gp_half(long nx, long ny, long nz, int which, double *u, double *v,
                    const double *V, double g, double dt, double dx, double dy, double dz) {
  const size_t sx = nx > 1 ? 1 : 0, sy = ny > 1 ? (size_t)nx : 0,
               sz = nz > 1 ? (size_t)nx * (size_t)ny : 0;
  double *out = which == 0 ? u : v;
  const double *w = which == 0 ? v : u;
#pragma omp parallel for schedule(static)
  for (long iz = LO(nz); iz < HI(nz); ++iz)
    for (long iy = LO(ny); iy < HI(ny); ++iy)
      for (long ix = LO(nx); ix < HI(nx); ++ix) {
        size_t p = AT(ix, iy, iz);
        double d2x = (w[p + sx] - w[p]) - (w[p] - w[p - sx]);
        double d2y = (w[p + sy] - w[p]) - (w[p] - w[p - sy]);
        double d2z = (w[p + sz] - w[p]) - (w[p] - w[p - sz]);
        double lap = ((d2x / (dx * dx)) + (d2y / (dy * dy))) + (d2z / (dz * dz));
        double h = -0.5 * lap + (V[p] + g * (u[p] * u[p] + v[p] * v[p])) * w[p];
        out[p] = which == 0 ? out[p] + dt * h : out[p] - dt * h;
      }
}

int oracle_threads(void) {
#ifdef _OPENMP
  int n = 1;
#pragma omp parallel
  {
#pragma omp single
    n = omp_get_num_threads();
  }
  return n;
#else
  return 1;
#endif
}

/* Set the number of OpenMP threads (no effect without OpenMP). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
