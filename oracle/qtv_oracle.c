/*
 * qtv_oracle.c -- plain, slow, FP64 CPU oracle for the two data-parallel
 * stages of vortex-core line vectorization:
 *
 *   (1) circulation-based vortex identification (Sec. 2.2.2, Eq. 5): the
 *       circulation C of the phase gradient around a closed grid path, which
 *       is 2*pi times an integer winding number when the path encloses a
 *       phase singularity and 0 otherwise;
 *   (2) density-guided sub-grid localization (Sec. 3.3.3, Eq. 6): the point
 *       x* = argmin rho(x), rho = |Phi|^2 (Eq. 3), with Phi linearly
 *       interpolated between grid nodes (Sec. 5, "Vectorization
 *       uncertainty"), restricted here to one pierced plaquette.
 *
 * TEST INFRASTRUCTURE ONLY.  The unit tests, the smoke check and the CPU
 * baseline leg of the benchmark are the only callers.  Nothing here is shared
 * with the CUDA path (no headers, helpers or constants in common).
 *
 * Every result is the plain definition written out in FP64, compiled with
 * -ffp-contract=off so that no fused multiply-add changes a rounding.
 *
 * Conventions (interface formats, not arithmetic):
 *   psi     complex64 interleaved (re, im), x fastest: node (i,j,k) is element
 *           (k*ny + j)*nx + i.
 *   face    named by its minimum corner (i,j,k) and an orientation o:
 *           o = 0: xy plaquette (normal +z), o = 1: yz (normal +x),
 *           o = 2: zx (normal +y).  Its corners, in loop order (counter-
 *           clockwise seen from the +normal side, i.e. right-handed about
 *           the normal), are
 *             o=0: (i,j,k) (i+1,j,k) (i+1,j+1,k) (i,j+1,k)
 *             o=1: (i,j,k) (i,j+1,k) (i,j+1,k+1) (i,j,k+1)
 *             o=2: (i,j,k) (i,j,k+1) (i+1,j,k+1) (i+1,j,k)
 *           A face exists iff its four corners lie in the grid (no
 *           periodic wrap).
 *   face id (lin << 2) | o with lin = (k*ny + j)*nx + i.
 *   dense arrays of per-face values are laid out [o][k][j][i].
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* per-face flag bits of the oracle */
#define OF_AMBIGUOUS 1u   /* an edge phase difference within 1e-4 rad of +-pi */
#define OF_ZERO_NODE 2u   /* a corner with psi == 0 exactly */
#define OF_NONFINITE 4u   /* a corner with a non-finite component */
#define OF_ABSENT 8u      /* face does not exist (a corner outside the grid) */
#define OF_RESIDUAL 16u   /* sum of edge phases not within 1e-9 of 2*pi*W */

/* per-sample flag bits of the localizer */
#define OL_ANOMALOUS 1u   /* |W| != 1, or no zero of the interpolant in the face */
#define OL_ILLCOND 2u     /* |det J| < 1e-3 * max|corner|^2 at the zero */

typedef struct {
  double re, im;
} ocplx;

static ocplx node_value(const float* psi, long nx, long ny, long i, long j, long k) {
  long idx = (k * ny + j) * nx + i;
  ocplx z;
  z.re = (double)psi[2 * idx];
  z.im = (double)psi[2 * idx + 1];
  return z;
}

static int is_finite_c(ocplx z) { return isfinite(z.re) && isfinite(z.im); }
static int is_zero_c(ocplx z) { return z.re == 0.0 && z.im == 0.0; }

/*
 * Wrapped phase difference along one directed grid edge a -> b: the discrete
 * form of the integrand of Eq. 5, grad(sigma).dl over one edge, taken as
 * arg(psi_b * conj(psi_a)) in (-pi, pi].
 *
 * Reading for a node with psi == 0 exactly (its phase is undefined): the node
 * is given phase 0, i.e. psi is replaced by 1 for this difference, and the
 * face is flagged OF_ZERO_NODE.
 */
static double edge_phase(ocplx a, ocplx b, unsigned* flags) {
  if (is_zero_c(a)) {
    a.re = 1.0;
    a.im = 0.0;
    *flags |= OF_ZERO_NODE;
  }
  if (is_zero_c(b)) {
    b.re = 1.0;
    b.im = 0.0;
    *flags |= OF_ZERO_NODE;
  }
  /* z = b * conj(a) */
  double zr = b.re * a.re + b.im * a.im;
  double zi = b.im * a.re - b.re * a.im;
  double d = atan2(zi, zr);
  if (OR_PI - fabs(d) < 1e-4) *flags |= OF_AMBIGUOUS;
  return d;
}

static void face_corners(const float* psi, long nx, long ny, long i, long j, long k, int o,
                         ocplx c[4]) {
  if (o == 0) {
    c[0] = node_value(psi, nx, ny, i, j, k);
    c[1] = node_value(psi, nx, ny, i + 1, j, k);
    c[2] = node_value(psi, nx, ny, i + 1, j + 1, k);
    c[3] = node_value(psi, nx, ny, i, j + 1, k);
  } else if (o == 1) {
    c[0] = node_value(psi, nx, ny, i, j, k);
    c[1] = node_value(psi, nx, ny, i, j + 1, k);
    c[2] = node_value(psi, nx, ny, i, j + 1, k + 1);
    c[3] = node_value(psi, nx, ny, i, j, k + 1);
  } else {
    c[0] = node_value(psi, nx, ny, i, j, k);
    c[1] = node_value(psi, nx, ny, i, j, k + 1);
    c[2] = node_value(psi, nx, ny, i + 1, j, k + 1);
    c[3] = node_value(psi, nx, ny, i + 1, j, k);
  }
}

static int face_exists(long nx, long ny, long nz, long i, long j, long k, int o) {
  if (o == 0) return i + 1 < nx && j + 1 < ny;
  if (o == 1) return j + 1 < ny && k + 1 < nz;
  return k + 1 < nz && i + 1 < nx;
}

/*
 * Winding number of one plaquette: Eq. 5 on the smallest closed grid path,
 * C = sum of the four wrapped edge phase differences in loop order, and
 * W = C / (2 pi) rounded to the nearest integer.  Faces that touch a
 * non-finite node get W = 0 and OF_NONFINITE.
 */
static int face_winding(const float* psi, long nx, long ny, long nz, long i, long j, long k,
                        int o, unsigned* flags, double* circ) {
  *flags = 0;
  *circ = 0.0;
  if (!face_exists(nx, ny, nz, i, j, k, o)) {
    *flags = OF_ABSENT;
    return 0;
  }
  ocplx c[4];
  face_corners(psi, nx, ny, i, j, k, o, c);
  for (int e = 0; e < 4; ++e)
    if (!is_finite_c(c[e])) {
      *flags = OF_NONFINITE;
      return 0;
    }
  double s = 0.0;
  for (int e = 0; e < 4; ++e) s += edge_phase(c[e], c[(e + 1) & 3], flags);
  double w = nearbyint(s / (2.0 * OR_PI));
  if (fabs(s - 2.0 * OR_PI * w) > 1e-9) *flags |= OF_RESIDUAL;
  *circ = s;
  return (int)w;
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Dense winding field for the planes k in [k0, k1) (all faces whose minimum
 * corner lies in those planes).  w and flags are [3][k1-k0][ny][nx]; circ
 * (optional, may be NULL) receives the FP64 circulation sum of each face.
 * Returns the number of faces with the OF_RESIDUAL flag (expected 0).
 */
long oracle_identify(int nx, int ny, int nz, int k0, int k1, const float* psi, int8_t* w,
                     uint8_t* flags, double* circ) {
  long nxl = nx, nyl = ny, nzl = nz;
  long nk = k1 - k0;
  long plane = nxl * nyl;
  long bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
  for (long kk = 0; kk < nk; ++kk) {
    long k = k0 + kk;
    for (int o = 0; o < 3; ++o)
      for (long j = 0; j < nyl; ++j)
        for (long i = 0; i < nxl; ++i) {
          unsigned f;
          double s;
          int wi = face_winding(psi, nxl, nyl, nzl, i, j, k, o, &f, &s);
          long out = ((long)o * nk + kk) * plane + j * nxl + i;
          w[out] = (int8_t)wi;
          flags[out] = (uint8_t)f;
          if (circ) circ[out] = s;
          if (f & OF_RESIDUAL) bad += 1;
        }
  }
  return bad;
}

/*
 * Node form of the circulation (Sec. 2.2.2, Fig. 2): for every grid node and
 * each of the three axis planes through it, the circulation along the ring
 * path made of the 8 grid edges of the 2h x 2h square centred on the node,
 * traversed in the same rotational sense as the plaquettes of that plane.
 * c_node is [3][nz][ny][nx] (plane index = orientation of the plaquettes that
 * tile the ring); nodes whose ring leaves the grid or touches a non-finite
 * value get 0.  vortex (optional) is [nz][ny][nx]: 1 where the maximum over the
 * three planes of |C| exceeds the threshold pi, else 0.
 */
void oracle_node_circulation(int nx, int ny, int nz, const float* psi, double* c_node,
                             uint8_t* vortex) {
  long nxl = nx, nyl = ny, nzl = nz;
  long vol = nxl * nyl * nzl;
#pragma omp parallel for schedule(dynamic, 1)
  for (long k = 0; k < nzl; ++k)
    for (long j = 0; j < nyl; ++j)
      for (long i = 0; i < nxl; ++i) {
        double best = 0.0;
        for (int o = 0; o < 3; ++o) {
          /* ring corners in the plane's (u, v) axes, counter-clockwise about
             the plane normal: (-1,-1) (1,-1) (1,1) (-1,1), 2 edges per side */
          /* u, v axis unit steps as (di,dj,dk) per orientation */
          long ua[3] = {0, 0, 0}, va[3] = {0, 0, 0};
          if (o == 0) { ua[0] = 1; va[1] = 1; }
          else if (o == 1) { ua[1] = 1; va[2] = 1; }
          else { ua[2] = 1; va[0] = 1; }
          static const int pu[9] = {-1, 0, 1, 1, 1, 0, -1, -1, -1};
          static const int pv[9] = {-1, -1, -1, 0, 1, 1, 1, 0, -1};
          int inside = 1;
          ocplx ring[8];
          for (int p = 0; p < 8 && inside; ++p) {
            long ii = i + pu[p] * ua[0] + pv[p] * va[0];
            long jj = j + pu[p] * ua[1] + pv[p] * va[1];
            long kk = k + pu[p] * ua[2] + pv[p] * va[2];
            if (ii < 0 || jj < 0 || kk < 0 || ii >= nxl || jj >= nyl || kk >= nzl) inside = 0;
            else {
              ring[p] = node_value(psi, nxl, nyl, ii, jj, kk);
              if (!is_finite_c(ring[p])) inside = 0;
            }
          }
          double s = 0.0;
          if (inside) {
            unsigned f = 0;
            for (int p = 0; p < 8; ++p) s += edge_phase(ring[p], ring[(p + 1) & 7], &f);
          }
          c_node[(long)o * vol + (k * nyl + j) * nxl + i] = s;
          if (fabs(s) > best) best = fabs(s);
        }
        if (vortex) vortex[(k * nyl + j) * nxl + i] = best > OR_PI ? 1 : 0;
      }
}

/* ---------------------------------------------------------------------------
 * Localization.  On a face with corners P0..P3 in loop order, placed at the
 * face-local coordinates (u,v) = (0,0) (1,0) (1,1) (0,1), the linearly
 * (bilinearly) interpolated field is
 *     F(u,v) = a + b u + c v + d u v,
 *     a = P0, b = P1 - P0, c = P3 - P0, d = P2 - P1 - P3 + P0.
 * Eq. 6 asks for argmin |F|^2 on the face; where W = +-1 the interpolant has
 * exactly one zero in the face, so the minimiser is that zero.  It is found
 * as a common root of Re F = 0 and Im F = 0: eliminating one coordinate
 * gives a quadratic in the other, solved in closed form, then each candidate
 * inside the face is refined by Newton's method and the one with the smallest
 * |F| is kept.
 * ------------------------------------------------------------------------- */

static ocplx cadd(ocplx x, ocplx y) { ocplx r = {x.re + y.re, x.im + y.im}; return r; }
static ocplx csub(ocplx x, ocplx y) { ocplx r = {x.re - y.re, x.im - y.im}; return r; }
static ocplx cscale(ocplx x, double s) { ocplx r = {x.re * s, x.im * s}; return r; }
/* Im(x * conj(y)) */
static double ccross(ocplx x, ocplx y) { return x.im * y.re - x.re * y.im; }
/* Re(x * conj(y)) */
static double cdotr(ocplx x, ocplx y) { return x.re * y.re + x.im * y.im; }
static double cabs2(ocplx x) { return x.re * x.re + x.im * x.im; }

static ocplx bilinear(const ocplx c[4], double u, double v) {
  ocplx r;
  double w0 = (1 - u) * (1 - v), w1 = u * (1 - v), w2 = u * v, w3 = (1 - u) * v;
  r.re = w0 * c[0].re + w1 * c[1].re + w2 * c[2].re + w3 * c[3].re;
  r.im = w0 * c[0].im + w1 * c[1].im + w2 * c[2].im + w3 * c[3].im;
  return r;
}

/* real roots of q2 t^2 + q1 t + q0 = 0; returns their number (0..2) */
static int real_roots(double q2, double q1, double q0, double t[2]) {
  double scale = fabs(q2) + fabs(q1) + fabs(q0);
  if (scale == 0.0) return 0;
  if (fabs(q2) <= 1e-14 * scale) {
    if (q1 == 0.0) return 0;
    t[0] = -q0 / q1;
    return 1;
  }
  double disc = q1 * q1 - 4.0 * q2 * q0;
  if (disc < 0.0) {
    if (disc > -1e-14 * q1 * q1) disc = 0.0;
    else return 0;
  }
  double sq = sqrt(disc);
  double qq = -0.5 * (q1 + (q1 >= 0 ? sq : -sq));
  if (qq == 0.0) {
    t[0] = 0.0;
    return 1;
  }
  t[0] = qq / q2;
  t[1] = q0 / qq;
  return 2;
}

/* Newton's method on (Re F, Im F) = 0 from (u,v); returns |F|^2 at the end */
static double newton_polish(const ocplx c[4], double* u, double* v) {
  ocplx a = c[0], b = csub(c[1], c[0]), cc = csub(c[3], c[0]);
  ocplx d = cadd(csub(csub(c[2], c[1]), c[3]), c[0]);
  double uu = *u, vv = *v;
  for (int it = 0; it < 20; ++it) {
    ocplx f = cadd(cadd(a, cscale(b, uu)), cadd(cscale(cc, vv), cscale(d, uu * vv)));
    ocplx fu = cadd(b, cscale(d, vv));
    ocplx fv = cadd(cc, cscale(d, uu));
    double det = fu.re * fv.im - fv.re * fu.im;
    if (det == 0.0) break;
    double du = -(fv.im * f.re - fv.re * f.im) / det;
    double dv = -(-fu.im * f.re + fu.re * f.im) / det;
    uu += du;
    vv += dv;
    if (fabs(du) + fabs(dv) < 1e-15) break;
  }
  *u = uu;
  *v = vv;
  return cabs2(bilinear(c, uu, vv));
}

/*
 * Localize one face.  Outputs (u, v), |F(u,v)|^2, the normalised Jacobian
 * determinant |det J| / max|corner|^2 at the result and the OL_* flags.
 * Returns 1 if a zero was found inside the face.
 */
static int localize_face(const ocplx c[4], int wind, double* uo, double* vo, double* resid,
                         double* detn, unsigned* flags) {
  ocplx a = c[0], b = csub(c[1], c[0]), cc = csub(c[3], c[0]);
  ocplx d = cadd(csub(csub(c[2], c[1]), c[3]), c[0]);
  double cand_u[4], cand_v[4];
  int nc = 0;
  double t[2];
  /* eliminate u: F = (a + cc v) + u (b + d v); u real <=> Im(p conj q) = 0 */
  int nr = real_roots(ccross(cc, d), ccross(a, d) + ccross(cc, b), ccross(a, b), t);
  for (int r = 0; r < nr; ++r) {
    double v = t[r];
    ocplx p = cadd(a, cscale(cc, v)), q = cadd(b, cscale(d, v));
    double qq = cabs2(q);
    if (qq == 0.0) continue;
    cand_u[nc] = -cdotr(p, q) / qq;
    cand_v[nc] = v;
    ++nc;
  }
  /* eliminate v: F = (a + b u) + v (cc + d u) */
  nr = real_roots(ccross(b, d), ccross(a, d) + ccross(b, cc), ccross(a, cc), t);
  for (int r = 0; r < nr; ++r) {
    double u = t[r];
    ocplx p = cadd(a, cscale(b, u)), q = cadd(cc, cscale(d, u));
    double qq = cabs2(q);
    if (qq == 0.0) continue;
    cand_u[nc] = u;
    cand_v[nc] = -cdotr(p, q) / qq;
    ++nc;
  }
  double m2 = 0.0;
  for (int e = 0; e < 4; ++e)
    if (cabs2(c[e]) > m2) m2 = cabs2(c[e]);
  const double tol = 1e-9;
  int found = 0;
  double best = INFINITY, bu = 0.5, bv = 0.5;
  for (int q = 0; q < nc; ++q) {
    double u = cand_u[q], v = cand_v[q];
    if (!(u >= -1e-6 && u <= 1 + 1e-6 && v >= -1e-6 && v <= 1 + 1e-6)) continue;
    double f2 = newton_polish(c, &u, &v);
    if (!(u >= -tol && u <= 1 + tol && v >= -tol && v <= 1 + tol)) continue;
    if (f2 < best) {
      best = f2;
      bu = u;
      bv = v;
      found = 1;
    }
  }
  *flags = 0;
  if (!found) {
    bu = 0.5;
    bv = 0.5;
    best = cabs2(bilinear(c, bu, bv));
  }
  if (!found || (wind != 1 && wind != -1)) *flags |= OL_ANOMALOUS;
  ocplx fu = cadd(b, cscale(d, bv)), fv = cadd(cc, cscale(d, bu));
  double det = fabs(fu.re * fv.im - fv.re * fu.im);
  *detn = m2 > 0 ? det / m2 : 0.0;
  if (*detn < 1e-3) *flags |= OL_ILLCOND;
  *uo = bu;
  *vo = bv;
  *resid = best;
  return found;
}

/*
 * Localize a list of faces (face ids as above, winding w per face).
 * Outputs per face: uv[2] (face-local coordinates), xyz[3] (position in
 * physical units: origin + h * grid coordinates), resid = |F(u,v)|^2,
 * detn = |det J| / max|corner|^2, flags (OL_*).  Returns the number of faces
 * for which no zero was found inside the face.
 */
long oracle_localize(int nx, int ny, int nz, const float* psi, long n, const uint64_t* face_ids,
                     const int8_t* w, double h, const double* origin, double* uv, double* xyz,
                     double* resid, double* detn, uint8_t* flags) {
  long nxl = nx, nyl = ny;
  long missing = 0;
  (void)nz;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : missing)
  for (long f = 0; f < n; ++f) {
    uint64_t id = face_ids[f];
    int o = (int)(id & 3u);
    long lin = (long)(id >> 2);
    long i = lin % nxl, j = (lin / nxl) % nyl, k = lin / (nxl * nyl);
    ocplx c[4];
    face_corners(psi, nxl, nyl, i, j, k, o, c);
    double u, v, r2, dn;
    unsigned fl;
    if (!localize_face(c, w[f], &u, &v, &r2, &dn, &fl)) missing += 1;
    double gx = (double)i, gy = (double)j, gz = (double)k;
    if (o == 0) { gx += u; gy += v; }
    else if (o == 1) { gy += u; gz += v; }
    else { gz += u; gx += v; }
    uv[2 * f] = u;
    uv[2 * f + 1] = v;
    xyz[3 * f] = origin[0] + h * gx;
    xyz[3 * f + 1] = origin[1] + h * gy;
    xyz[3 * f + 2] = origin[2] + h * gz;
    resid[f] = r2;
    detn[f] = dn;
    flags[f] = (uint8_t)fl;
  }
  return missing;
}

/*
 * Linearly (trilinearly) interpolated density rho(x) = |Phi(x)|^2 at
 * arbitrary points in grid coordinates (Eq. 3 with the interpolation
 * assumption of Sec. 5); used for the density error metric of Eq. 7.
 * Points outside the grid get NAN.
 */
void oracle_density(int nx, int ny, int nz, const float* psi, long n, const double* p,
                    double* rho) {
  long nxl = nx, nyl = ny, nzl = nz;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < n; ++q) {
    double x = p[3 * q], y = p[3 * q + 1], z = p[3 * q + 2];
    if (!(x >= 0 && y >= 0 && z >= 0 && x <= nxl - 1 && y <= nyl - 1 && z <= nzl - 1)) {
      rho[q] = NAN;
      continue;
    }
    long i = (long)floor(x), j = (long)floor(y), k = (long)floor(z);
    if (i > nxl - 2) i = nxl - 2;
    if (j > nyl - 2) j = nyl - 2;
    if (k > nzl - 2) k = nzl - 2;
    if (i < 0) i = 0;
    if (j < 0) j = 0;
    if (k < 0) k = 0;
    double fx = x - i, fy = y - j, fz = z - k;
    ocplx acc = {0.0, 0.0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          long ii = i + dx < nxl ? i + dx : i, jj = j + dy < nyl ? j + dy : j,
               kk = k + dz < nzl ? k + dz : k;
          double wgt = (dx ? fx : 1 - fx) * (dy ? fy : 1 - fy) * (dz ? fz : 1 - fz);
          ocplx val = node_value(psi, nxl, nyl, ii, jj, kk);
          acc.re += wgt * val.re;
          acc.im += wgt * val.im;
        }
    rho[q] = cabs2(acc);
  }
}

/* ---------------------------------------------------------------------------
 * Sample refinement (Sec. 3.3.3, "Locating more accurate sample points"): an
 * initial estimate x0 of a core sample (the paper uses the box means of the
 * graph reduction) is moved to a minimizer of rho = |psi|^2 (Eq. 6) within
 * the plane through x0 perpendicular to the local core direction t, which the
 * paper takes from the pseudo-vorticity of Rorai et al.:
 *   t = grad Re psi x grad Im psi at x0, normalized.
 * Readings where the paper is silent:
 *   - psi between nodes is the trilinear interpolant (Sec. 5: linearly
 *     interpolated); rho and its gradient are those of that interpolant,
 *     the gradient taken within the cell floor(x) (index clamped to
 *     [0, n - 2], as in oracle_density);
 *   - grad Re psi and grad Im psi at x0 are the node gradients by central
 *     differences (one-sided on the boundary, 0 along an axis of one node)
 *     interpolated trilinearly;
 *   - gradient descent on the in-plane gradient g = grad rho - (grad rho . t) t;
 *     each step starts at alpha = 2 rho / |g|^2 (the exact step for a round
 *     bowl whose minimum is 0) and halves alpha until the Armijo condition
 *     rho(x - alpha g) <= rho(x) - 1e-4 alpha |g|^2 holds with the new point
 *     inside the grid and inside the box |x - x0|_inf <= 1 (grid units); a
 *     step that would leave either is rejected, not projected, so a result on
 *     the grid or box boundary is a constrained stop;
 *   - it stops, converged, when no step of length >= tol decreases rho that
 *     way (or g = 0), or after max_iter accepted steps.
 * Per sample: x, rho(x), t, the determinant of the 2x2 real Jacobian of psi
 * with respect to in-plane coordinates (e1, e2) at x (conditioning), the
 * number of steps taken, and flags: 1 converged, 2 no tangent (the cross
 * product is zero or x0 lies outside the grid: x = x0), 4 step limit.
 * ------------------------------------------------------------------------- */
#define OR_CONVERGED 1u
#define OR_NO_TANGENT 2u
#define OR_MAX_ITER 4u

/* cell of x along an axis of n nodes: floor(x) clamped to [0, n-2] (0 if n < 2) */
static long cell_of(double x, long n) {
  long i = (long)floor(x);
  if (i > n - 2) i = n - 2;
  if (i < 0) i = 0;
  return i;
}

static int inside_grid(const double x[3], long nx, long ny, long nz) {
  return x[0] >= 0 && x[1] >= 0 && x[2] >= 0 && x[0] <= nx - 1 && x[1] <= ny - 1 &&
         x[2] <= nz - 1;
}

/* trilinear psi at x and its partial derivatives d[0..2] within cell floor(x) */
static ocplx trilinear_eval(const float* psi, long nx, long ny, long nz, const double x[3],
                            ocplx d[3]) {
  const long i = cell_of(x[0], nx), j = cell_of(x[1], ny), k = cell_of(x[2], nz);
  const double f[3] = {x[0] - i, x[1] - j, x[2] - k};
  const long base[3] = {i, j, k}, n[3] = {nx, ny, nz};
  ocplx acc = {0.0, 0.0};
  for (int a = 0; a < 3; ++a) d[a].re = d[a].im = 0.0;
  for (int c = 0; c < 8; ++c) {
    long idx[3];
    double w[3], dw[3];
    for (int a = 0; a < 3; ++a) {
      const int bit = (c >> a) & 1;
      idx[a] = base[a] + bit < n[a] ? base[a] + bit : base[a];
      w[a] = bit ? f[a] : 1.0 - f[a];
      dw[a] = bit ? 1.0 : -1.0;
    }
    const ocplx v = node_value(psi, nx, ny, idx[0], idx[1], idx[2]);
    const double wt = w[0] * w[1] * w[2];
    acc.re += wt * v.re;
    acc.im += wt * v.im;
    const double dd[3] = {dw[0] * w[1] * w[2], w[0] * dw[1] * w[2], w[0] * w[1] * dw[2]};
    for (int a = 0; a < 3; ++a) {
      d[a].re += dd[a] * v.re;
      d[a].im += dd[a] * v.im;
    }
  }
  return acc;
}

/* central-difference gradient of psi at node (i,j,k) along axis a */
static ocplx node_grad(const float* psi, long nx, long ny, long nz, long i, long j, long k, int a) {
  const long n[3] = {nx, ny, nz};
  long p[3] = {i, j, k}, q[3] = {i, j, k};
  double s = 0.5;
  if (n[a] < 2) {
    ocplx z = {0.0, 0.0};
    return z;
  }
  if (p[a] == 0) {
    q[a] = 1;
    s = 1.0;
  } else if (p[a] == n[a] - 1) {
    p[a] = n[a] - 2;
    s = 1.0;
  } else {
    p[a] -= 1;
    q[a] += 1;
  }
  const ocplx lo = node_value(psi, nx, ny, p[0], p[1], p[2]);
  const ocplx hi = node_value(psi, nx, ny, q[0], q[1], q[2]);
  return cscale(csub(hi, lo), s);
}

/* pseudo-vorticity direction at x: interpolated node gradients, cross product */
static void pseudo_vorticity(const float* psi, long nx, long ny, long nz, const double x[3],
                             double t[3]) {
  const long i = cell_of(x[0], nx), j = cell_of(x[1], ny), k = cell_of(x[2], nz);
  const double f[3] = {x[0] - i, x[1] - j, x[2] - k};
  const long base[3] = {i, j, k}, n[3] = {nx, ny, nz};
  double gr[3] = {0, 0, 0}, gi[3] = {0, 0, 0};
  for (int c = 0; c < 8; ++c) {
    long idx[3];
    double wt = 1.0;
    for (int a = 0; a < 3; ++a) {
      const int bit = (c >> a) & 1;
      idx[a] = base[a] + bit < n[a] ? base[a] + bit : base[a];
      wt *= bit ? f[a] : 1.0 - f[a];
    }
    for (int a = 0; a < 3; ++a) {
      const ocplx g = node_grad(psi, nx, ny, nz, idx[0], idx[1], idx[2], a);
      gr[a] += wt * g.re;
      gi[a] += wt * g.im;
    }
  }
  t[0] = gr[1] * gi[2] - gr[2] * gi[1];
  t[1] = gr[2] * gi[0] - gr[0] * gi[2];
  t[2] = gr[0] * gi[1] - gr[1] * gi[0];
}

static double rho_at(const float* psi, long nx, long ny, long nz, const double x[3],
                     double grad[3]) {
  ocplx d[3];
  const ocplx v = trilinear_eval(psi, nx, ny, nz, x, d);
  for (int a = 0; a < 3; ++a) grad[a] = 2.0 * (v.re * d[a].re + v.im * d[a].im);
  return cabs2(v);
}

void oracle_refine(int nx, int ny, int nz, const float* psi, long n, const double* x0s,
                   int max_iter, double tol, double* xout, double* rho_out, double* tang,
                   double* detj, int32_t* iters, uint8_t* flags) {
  const long NX = nx, NY = ny, NZ = nz;
#pragma omp parallel for schedule(dynamic, 16)
  for (long q = 0; q < n; ++q) {
    const double* x0 = x0s + 3 * q;
    double x[3] = {x0[0], x0[1], x0[2]}, t[3] = {0, 0, 0}, grad[3];
    unsigned fl = 0;
    int it = 0;
    double rho = NAN, dj = 0.0;
    if (!inside_grid(x0, NX, NY, NZ)) {
      fl = OR_NO_TANGENT;
    } else {
      pseudo_vorticity(psi, NX, NY, NZ, x0, t);
      const double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
      rho = rho_at(psi, NX, NY, NZ, x, grad);
      if (!(tn > 0.0) || !isfinite(tn)) {
        fl = OR_NO_TANGENT;
      } else {
        for (int a = 0; a < 3; ++a) t[a] /= tn;
        fl = OR_MAX_ITER;
        for (it = 0; it < max_iter;) {
          const double gt = grad[0] * t[0] + grad[1] * t[1] + grad[2] * t[2];
          double g[3];
          for (int a = 0; a < 3; ++a) g[a] = grad[a] - gt * t[a];
          const double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
          if (!(gg > 0.0)) {
            fl = OR_CONVERGED;
            break;
          }
          const double gn = sqrt(gg);
          double alpha = 2.0 * rho / gg;
          int accepted = 0;
          double xn[3], rn = 0.0, gnext[3];
          while (alpha * gn >= tol) {
            for (int a = 0; a < 3; ++a) xn[a] = x[a] - alpha * g[a];
            if (inside_grid(xn, NX, NY, NZ) && fabs(xn[0] - x0[0]) <= 1.0 &&
                fabs(xn[1] - x0[1]) <= 1.0 && fabs(xn[2] - x0[2]) <= 1.0) {
              rn = rho_at(psi, NX, NY, NZ, xn, gnext);
              if (rn <= rho - 1e-4 * alpha * gg) {
                accepted = 1;
                break;
              }
            }
            alpha *= 0.5;
          }
          if (!accepted) {
            fl = OR_CONVERGED;
            break;
          }
          ++it;
          for (int a = 0; a < 3; ++a) {
            x[a] = xn[a];
            grad[a] = gnext[a];
          }
          rho = rn;
        }
      }
    }
    if (!(fl & OR_NO_TANGENT)) {
      /* in-plane Jacobian of psi at x: basis e1 = normalize(t x a), e2 = t x e1
         with a the coordinate axis least aligned with t */
      int m = 0;
      for (int a = 1; a < 3; ++a)
        if (fabs(t[a]) < fabs(t[m])) m = a;
      double ax[3] = {0, 0, 0};
      ax[m] = 1.0;
      double e1[3] = {t[1] * ax[2] - t[2] * ax[1], t[2] * ax[0] - t[0] * ax[2],
                      t[0] * ax[1] - t[1] * ax[0]};
      const double en = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
      for (int a = 0; a < 3; ++a) e1[a] /= en;
      const double e2[3] = {t[1] * e1[2] - t[2] * e1[1], t[2] * e1[0] - t[0] * e1[2],
                            t[0] * e1[1] - t[1] * e1[0]};
      ocplx d[3];
      (void)trilinear_eval(psi, NX, NY, NZ, x, d);
      double a1r = 0, a1i = 0, a2r = 0, a2i = 0;
      for (int a = 0; a < 3; ++a) {
        a1r += d[a].re * e1[a];
        a1i += d[a].im * e1[a];
        a2r += d[a].re * e2[a];
        a2i += d[a].im * e2[a];
      }
      dj = a1r * a2i - a2r * a1i;
    }
    for (int a = 0; a < 3; ++a) {
      xout[3 * q + a] = x[a];
      if (tang) tang[3 * q + a] = t[a];
    }
    if (rho_out) rho_out[q] = rho;
    if (detj) detj[q] = dj;
    if (iters) iters[q] = it;
    flags[q] = (uint8_t)fl;
  }
}
