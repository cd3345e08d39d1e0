/*
 * fv_oracle.c -- plain, slow FP64 reference of the cell-centred finite-volume
 * Euler step on triangles (Nagy et al., "Accelerating unstructured finite
 * volume computations on field-programmable gate arrays", Sec. 6).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header or constant table with the
 * CUDA library: every formula below is written out again from the paper.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared fv_oracle.c -lm
 * (-ffp-contract=off keeps each operation rounded as written.)
 *
 * Conventions (the input format the library also accepts):
 *   state     U[c*4 + {0,1,2,3}] = (rho, rho*u, rho*v, E)          Sec. 6.1
 *   triangle  tri[c*3 + k] node ids; face k runs from vertex k to k+1 (mod 3)
 *   nbr       nbr[c*3 + k] >= 0: the cell across face k;
 *             -1 slip wall, -2 far field (free-stream ghost), -3 extrapolation
 *   normals   nrm[c*6 + 2k + {0,1}] outward normal of face k scaled by the
 *             face length (Sec. 6.2.1)
 *   vol       vol[c] triangle area V_T (Sec. 6.2.1)
 *   boundary  bnd[j*3 + {0,1,2}] = (node a, node b, tag), tag 1 wall,
 *             2 far field, 3 extrapolation
 *
 * Readings of the paper taken here (the paper is silent or inconsistent):
 *   R0  the dissipation enters with the minus sign of Eq. 5; Eq. 7a-7d print
 *       a plus, which makes the scheme anti-dissipative.
 *   R1  the time step is not given by the paper; dt = CFL * min_T
 *       2 V_T / (P_T (|v_T| + c_T)), P_T the perimeter, evaluated on U^n.
 *       cfl < 0 means a fixed step dt = -cfl.
 *   R2  |u-bar| is the absolute value of the mean of the two face-normal
 *       velocities, c-bar the mean of the two sound speeds (Eq. 5 text).
 *   R3  ghost cells: wall mirrors the normal momentum, far field is the
 *       free stream, extrapolation copies the interior state.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GAMMA 1.4 /* ratio of specific heats, Sec. 6.1 after Eq. 2 */

#define ORC_WALL (-1)
#define ORC_FARFIELD (-2)
#define ORC_EXTRAP (-3)

/* error codes returned by orc_build_mesh */
#define ORC_OK 0
#define ORC_E_DEGENERATE (-1)
#define ORC_E_NONMANIFOLD (-2)
#define ORC_E_OPEN_EDGE (-3)
#define ORC_E_COLLAPSED (-4)
#define ORC_E_NOMEM (-5)
#define ORC_E_BADINPUT (-6)

/* ------------------------------------------------------------------------ */
/* Mesh geometry (Sec. 6.2.1) and neighbour search (Sec. 7: every triangle  */
/* has three neighbours, ghost cells at the boundary).                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t a, b; /* canonical node ids, a < b */
  int64_t cell;
  int32_t face;
} orc_edge;

static int orc_edge_cmp(const void* pa, const void* pb) {
  const orc_edge* x = (const orc_edge*)pa;
  const orc_edge* y = (const orc_edge*)pb;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
  return x->face - y->face;
}

static double orc_signed_area(const double* xy, int32_t i0, int32_t i1, int32_t i2) {
  double ax = xy[2 * i1] - xy[2 * i0], ay = xy[2 * i1 + 1] - xy[2 * i0 + 1];
  double bx = xy[2 * i2] - xy[2 * i0], by = xy[2 * i2 + 1] - xy[2 * i0 + 1];
  return 0.5 * (ax * by - bx * ay);
}

/* Builds neighbours, outward scaled normals and areas.  Triangles given
 * clockwise are reoriented.  canon (nullable) maps a node to the node it is
 * identified with on a periodic domain.  Sec. 7 precomputes the size and
 * normal of every face: each face gets one normal, computed from the
 * coordinates of one of its two cells, and the other cell uses its negation.
 * The two copies of a periodic face differ in their node coordinates by
 * rounding, so the cell that supplies the coordinates is fixed by node ids
 * alone: the side whose (smaller, larger) raw node-id pair of the edge is the
 * smaller pair. */
int orc_build_mesh(int64_t n_nodes, const double* xy, int64_t n_tri, const int32_t* tri,
                   const int32_t* canon, int64_t n_bnd, const int32_t* bnd,
                   int32_t default_bc, int32_t* nbr, double* nrm, double* vol) {
  int64_t c, j;
  int k;
  if (n_tri < 0 || n_nodes < 0) return ORC_E_BADINPUT;
  for (j = 0; j < 3 * n_tri; ++j)
    if (tri[j] < 0 || tri[j] >= n_nodes) return ORC_E_BADINPUT;
  orc_edge* e = (orc_edge*)malloc(sizeof(orc_edge) * (size_t)(3 * n_tri + 1));
  orc_edge* be = (orc_edge*)malloc(sizeof(orc_edge) * (size_t)(n_bnd + 1));
  int32_t* vt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(3 * n_tri + 1));
  if (!e || !be || !vt) {
    free(e);
    free(be);
    free(vt);
    return ORC_E_NOMEM;
  }
  for (c = 0; c < n_tri; ++c) {
    int32_t v[3] = {tri[3 * c], tri[3 * c + 1], tri[3 * c + 2]};
    double area = orc_signed_area(xy, v[0], v[1], v[2]);
    if (area == 0.0 || !isfinite(area)) {
      free(e);
      free(be);
      free(vt);
      return ORC_E_DEGENERATE;
    }
    if (area < 0.0) { /* make the vertex order counter-clockwise */
      int32_t t = v[1];
      v[1] = v[2];
      v[2] = t;
      area = -area;
    }
    vol[c] = area;
    vt[3 * c] = v[0];
    vt[3 * c + 1] = v[1];
    vt[3 * c + 2] = v[2];
    for (k = 0; k < 3; ++k) {
      int32_t p = v[k], q = v[(k + 1) % 3];
      /* outward normal of edge p->q on a CCW triangle, scaled by |pq| */
      nrm[6 * c + 2 * k] = xy[2 * q + 1] - xy[2 * p + 1];
      nrm[6 * c + 2 * k + 1] = -(xy[2 * q] - xy[2 * p]);
      int64_t ca = canon ? canon[p] : p, cb = canon ? canon[q] : q;
      if (ca == cb) {
        free(e);
        free(be);
        free(vt);
        return ORC_E_COLLAPSED;
      }
      e[3 * c + k].a = ca < cb ? ca : cb;
      e[3 * c + k].b = ca < cb ? cb : ca;
      e[3 * c + k].cell = c;
      e[3 * c + k].face = k;
    }
  }
  for (j = 0; j < n_bnd; ++j) {
    int64_t ca = canon ? canon[bnd[3 * j]] : bnd[3 * j];
    int64_t cb = canon ? canon[bnd[3 * j + 1]] : bnd[3 * j + 1];
    be[j].a = ca < cb ? ca : cb;
    be[j].b = ca < cb ? cb : ca;
    be[j].cell = bnd[3 * j + 2];
    be[j].face = 0;
  }
  qsort(e, (size_t)(3 * n_tri), sizeof(orc_edge), orc_edge_cmp);
  qsort(be, (size_t)n_bnd, sizeof(orc_edge), orc_edge_cmp);
  j = 0;
  while (j < 3 * n_tri) {
    int64_t m = j + 1;
    while (m < 3 * n_tri && e[m].a == e[j].a && e[m].b == e[j].b) ++m;
    if (m - j > 2) {
      free(e);
      free(be);
      free(vt);
      return ORC_E_NONMANIFOLD;
    }
    if (m - j == 2) {
      int64_t s0 = 3 * e[j].cell + e[j].face, s1 = 3 * e[j + 1].cell + e[j + 1].face;
      nbr[s0] = (int32_t)e[j + 1].cell;
      nbr[s1] = (int32_t)e[j].cell;
      /* one normal per face: the owner side keeps its own, the other negates it */
      int32_t a0 = vt[s0], b0 = vt[3 * e[j].cell + (e[j].face + 1) % 3];
      int32_t a1 = vt[s1], b1 = vt[3 * e[j + 1].cell + (e[j + 1].face + 1) % 3];
      int32_t lo0 = a0 < b0 ? a0 : b0, hi0 = a0 < b0 ? b0 : a0;
      int32_t lo1 = a1 < b1 ? a1 : b1, hi1 = a1 < b1 ? b1 : a1;
      int own0 = lo0 < lo1 || (lo0 == lo1 && hi0 <= hi1);
      int64_t own = own0 ? s0 : s1, other = own0 ? s1 : s0;
      nrm[2 * other] = -nrm[2 * own];
      nrm[2 * other + 1] = -nrm[2 * own + 1];
    } else {
      int32_t tag = default_bc;
      int64_t lo = 0, hi = n_bnd; /* binary search of the boundary list */
      while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (be[mid].a < e[j].a || (be[mid].a == e[j].a && be[mid].b < e[j].b))
          lo = mid + 1;
        else
          hi = mid;
      }
      if (lo < n_bnd && be[lo].a == e[j].a && be[lo].b == e[j].b) tag = (int32_t)be[lo].cell;
      if (tag < 1 || tag > 3) {
        free(e);
        free(be);
        free(vt);
        return ORC_E_OPEN_EDGE;
      }
      nbr[3 * e[j].cell + e[j].face] = -tag;
    }
    j = m;
  }
  free(e);
  free(be);
  free(vt);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Thermodynamics (Eq. 2 and the sound speed defined after it).             */
/* ------------------------------------------------------------------------ */

static double orc_pressure(const double* U) {
  double u = U[1] / U[0], v = U[2] / U[0];
  return (ORC_GAMMA - 1.0) * (U[3] - 0.5 * U[0] * (u * u + v * v));
}

static double orc_sound_speed(double rho, double p) { return sqrt(ORC_GAMMA * p / rho); }

/* Ghost state across a boundary face (reading R3). */
void orc_ghost(int32_t code, const double* UL, const double* n, const double* uinf, double* UR) {
  if (code == ORC_WALL) {
    double len = sqrt(n[0] * n[0] + n[1] * n[1]);
    double nx = n[0] / len, ny = n[1] / len;
    double mn = UL[1] * nx + UL[2] * ny;
    UR[0] = UL[0];
    UR[1] = UL[1] - 2.0 * mn * nx;
    UR[2] = UL[2] - 2.0 * mn * ny;
    UR[3] = UL[3];
  } else if (code == ORC_FARFIELD) {
    memcpy(UR, uinf, 4 * sizeof(double));
  } else {
    memcpy(UR, UL, 4 * sizeof(double));
  }
}

/* ------------------------------------------------------------------------ */
/* Lax-Friedrichs flux across one face, in the face frame (Eq. 5, Eq. 7a-7d */
/* with reading R0), rotated back to x-y by R_n (update equation, Sec.      */
/* 6.2.2) and multiplied by the face length |n|.  s scales the dissipation  */
/* (s = 1 is the paper's flux; other values come from the learned closure). */
/* ------------------------------------------------------------------------ */

typedef struct {
  double rho, mn, mt, E; /* conserved state in the face frame */
  double un, ut, p, c;   /* face-normal and tangential velocity, pressure, sound speed */
} orc_face_state;

static void orc_to_face_frame(const double* U, double nx, double ny, orc_face_state* s) {
  s->rho = U[0];
  s->mn = U[1] * nx + U[2] * ny;    /* x-axis of the face frame: the unit normal */
  s->mt = -U[1] * ny + U[2] * nx;   /* y-axis: the unit tangent (-ny, nx) */
  s->E = U[3];
  s->un = s->mn / s->rho;
  s->ut = s->mt / s->rho;
  s->p = (ORC_GAMMA - 1.0) * (s->E - 0.5 * s->rho * (s->un * s->un + s->ut * s->ut));
  s->c = orc_sound_speed(s->rho, s->p);
}

/* Wave speed of the dissipation: 0 = the paper's interface averages (reading */
/* R2), 1 = the larger one-sided |u_n| + c (Rusanov), an alternative reading  */
/* of the same passage kept for sensitivity checks.  Process-wide setting.    */
static int orc_wave_mode = 0;

void orc_set_wave_speed(int32_t mode) { orc_wave_mode = mode; }

void orc_face_flux(const double* UL, const double* UR, const double* n, double scale, double* F) {
  double len = sqrt(n[0] * n[0] + n[1] * n[1]);
  double nx = n[0] / len, ny = n[1] / len;
  orc_face_state L, R;
  orc_to_face_frame(UL, nx, ny, &L);
  orc_to_face_frame(UR, nx, ny, &R);
  double ubar = 0.5 * (L.un + R.un);
  double cbar = 0.5 * (L.c + R.c);
  double a;
  if (orc_wave_mode == 0) {
    a = scale * (fabs(ubar) + cbar);
  } else {
    double aL = fabs(L.un) + L.c, aR = fabs(R.un) + R.c;
    a = scale * (aL > aR ? aL : aR);
  }
  /* Eq. 7a-7d, face frame */
  double f_rho = 0.5 * (L.rho * L.un + R.rho * R.un) - 0.5 * a * (R.rho - L.rho);
  double f_mn = 0.5 * ((L.rho * L.un * L.un + L.p) + (R.rho * R.un * R.un + R.p)) -
                0.5 * a * (R.mn - L.mn);
  double f_mt = 0.5 * (L.rho * L.un * L.ut + R.rho * R.un * R.ut) - 0.5 * a * (R.mt - L.mt);
  double f_E = 0.5 * ((L.E + L.p) * L.un + (R.E + R.p) * R.un) - 0.5 * a * (R.E - L.E);
  /* rotate back with R_n and scale by |n| */
  F[0] = len * f_rho;
  F[1] = len * (f_mn * nx - f_mt * ny);
  F[2] = len * (f_mn * ny + f_mt * nx);
  F[3] = len * f_E;
}

/* ------------------------------------------------------------------------ */
/* Learned dissipation scale (not in the paper): an MLP 8 -> 32 -> 32 -> 1   */
/* with ReLU, s = 0.2 + 1.3 sigmoid(z).  Parameter vector theta, flat:      */
/*   W1[32][8], b1[32], W2[32][32], b2[32], w3[32], b3                      */
/* Optional rounding of the layer inputs to bfloat16 (round to nearest      */
/* even) models tensor-core operands.                                        */
/* ------------------------------------------------------------------------ */

#define ORC_NF 8
#define ORC_NH 32
#define ORC_OFF_W1 0
#define ORC_OFF_B1 (ORC_OFF_W1 + ORC_NH * ORC_NF)
#define ORC_OFF_W2 (ORC_OFF_B1 + ORC_NH)
#define ORC_OFF_B2 (ORC_OFF_W2 + ORC_NH * ORC_NH)
#define ORC_OFF_W3 (ORC_OFF_B2 + ORC_NH)
#define ORC_OFF_B3 (ORC_OFF_W3 + ORC_NH)
#define ORC_NPARAM (ORC_OFF_B3 + 1)

int64_t orc_closure_nparam(void) { return ORC_NPARAM; }

/* bfloat16 round-to-nearest-even of a float, returned as double */
static double orc_round_bf16(double x) {
  float f = (float)x;
  uint32_t b;
  memcpy(&b, &f, 4);
  if ((b & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf/nan unchanged */
  uint32_t lsb = (b >> 16) & 1u;
  b += 0x7fffu + lsb;
  b &= 0xffff0000u;
  memcpy(&f, &b, 4);
  return (double)f;
}

/* Eight features of a face that do not change when L and R are swapped and n
 * is negated, so the scale is the same seen from both cells (flux stays
 * antisymmetric, the scheme stays conservative). */
void orc_closure_features(const double* UL, const double* UR, const double* n, double* f) {
  double len = sqrt(n[0] * n[0] + n[1] * n[1]);
  double nx = n[0] / len, ny = n[1] / len;
  orc_face_state L, R;
  orc_to_face_frame(UL, nx, ny, &L);
  orc_to_face_frame(UR, nx, ny, &R);
  double rbar = 0.5 * (L.rho + R.rho);
  double pbar = 0.5 * (L.p + R.p);
  double cbar = 0.5 * (L.c + R.c);
  f[0] = fabs(R.rho - L.rho) / rbar;
  f[1] = fabs(R.un - L.un) / cbar;
  f[2] = fabs(R.ut - L.ut) / cbar;
  f[3] = fabs(R.p - L.p) / pbar;
  f[4] = fabs(0.5 * (L.un + R.un)) / cbar;
  f[5] = fabs(R.un / R.c - L.un / L.c);
  f[6] = (L.c < R.c ? L.c : R.c) / cbar;
  f[7] = (L.c < R.c ? R.c : L.c) / cbar;
}

typedef struct {
  double x[ORC_NF];
  double a1[ORC_NH], h1[ORC_NH];
  double a2[ORC_NH], h2[ORC_NH];
  double z, sig, s;
} orc_mlp_trace;

static void orc_mlp_forward(const double* th, const double* feat, int bf16_acts, orc_mlp_trace* t) {
  int i, j;
  for (j = 0; j < ORC_NF; ++j) t->x[j] = bf16_acts ? orc_round_bf16(feat[j]) : feat[j];
  for (i = 0; i < ORC_NH; ++i) {
    double acc = th[ORC_OFF_B1 + i];
    for (j = 0; j < ORC_NF; ++j) acc += th[ORC_OFF_W1 + i * ORC_NF + j] * t->x[j];
    t->a1[i] = acc;
    t->h1[i] = acc > 0.0 ? acc : 0.0;
    if (bf16_acts) t->h1[i] = orc_round_bf16(t->h1[i]);
  }
  for (i = 0; i < ORC_NH; ++i) {
    double acc = th[ORC_OFF_B2 + i];
    for (j = 0; j < ORC_NH; ++j) acc += th[ORC_OFF_W2 + i * ORC_NH + j] * t->h1[j];
    t->a2[i] = acc;
    t->h2[i] = acc > 0.0 ? acc : 0.0;
  }
  double z = th[ORC_OFF_B3];
  for (j = 0; j < ORC_NH; ++j) z += th[ORC_OFF_W3 + j] * t->h2[j];
  t->z = z;
  t->sig = 1.0 / (1.0 + exp(-z));
  t->s = 0.2 + 1.3 * t->sig;
}

/* Accumulates d(loss)/d(theta) given d(loss)/d(s) for one evaluation. */
static void orc_mlp_backward(const double* th, const orc_mlp_trace* t, double gs, double* grad) {
  int i, j;
  double dz = gs * 1.3 * t->sig * (1.0 - t->sig);
  double d2[ORC_NH], d1[ORC_NH];
  grad[ORC_OFF_B3] += dz;
  for (j = 0; j < ORC_NH; ++j) {
    grad[ORC_OFF_W3 + j] += dz * t->h2[j];
    d2[j] = t->a2[j] > 0.0 ? dz * th[ORC_OFF_W3 + j] : 0.0;
  }
  for (i = 0; i < ORC_NH; ++i) {
    grad[ORC_OFF_B2 + i] += d2[i];
    for (j = 0; j < ORC_NH; ++j) grad[ORC_OFF_W2 + i * ORC_NH + j] += d2[i] * t->h1[j];
  }
  for (j = 0; j < ORC_NH; ++j) {
    double acc = 0.0;
    for (i = 0; i < ORC_NH; ++i) acc += th[ORC_OFF_W2 + i * ORC_NH + j] * d2[i];
    d1[j] = t->a1[j] > 0.0 ? acc : 0.0;
  }
  for (i = 0; i < ORC_NH; ++i) {
    grad[ORC_OFF_B1 + i] += d1[i];
    for (j = 0; j < ORC_NF; ++j) grad[ORC_OFF_W1 + i * ORC_NF + j] += d1[i] * t->x[j];
  }
}

/* The MLP alone on a given feature vector (the features rounded to
 * bfloat16 first when bf16_acts). */
double orc_closure_mlp(const double* theta, int32_t bf16_acts, const double* feat) {
  orc_mlp_trace t;
  orc_mlp_forward(theta, feat, bf16_acts, &t);
  return t.s;
}

double orc_closure_scale(const double* theta, int32_t bf16_acts, const double* UL,
                         const double* UR, const double* n) {
  double f[ORC_NF];
  orc_mlp_trace t;
  orc_closure_features(UL, UR, n, f);
  orc_mlp_forward(theta, f, bf16_acts, &t);
  return t.s;
}

/* ------------------------------------------------------------------------ */
/* Rounding ambiguity of the learned scale (test support).                  */
/*                                                                          */
/* A device evaluates the features in FP32 and the first hidden layer with  */
/* FP32 accumulation, then rounds both to bfloat16 as tensor-core operands.  */
/* Where such a value lies within its FP32 evaluation error of a bfloat16    */
/* rounding boundary, either neighbouring bfloat16 value is a correct       */
/* result of that evaluation, and the scale differs accordingly (a relative */
/* change of up to 2^-8 in one operand).  The functions below bound the     */
/* FP32 evaluation error of every rounded value and enumerate the scales of */
/* all admissible roundings, so that a device result can be checked        */
/* against the set instead of against one value.                           */
/* ------------------------------------------------------------------------ */

static void orc_neighbour_state(int64_t c, int k, const int32_t* nbr, const double* nrm,
                                const double* uinf, const double* U, double* UR);

/* Relative error bound of one FP32 operation, taken as 2^-22 so that it    */
/* also covers approximate reciprocals and square roots (about 2^-23).      */
#define ORC_U32 (1.0 / 8388608.0)
/* Safety factor on the first-order error bounds below. */
#define ORC_ERR_SAFETY 1.0

/* First-order bounds on |f32 - f| for the eight features of
 * orc_closure_features evaluated in FP32 from the same (FP32-exact) states:
 * each operation is charged ORC_U32 of its result and the errors of its
 * inputs are propagated by their partial derivatives.  err[8] out. */
void orc_closure_feature_errors(const double* UL, const double* UR, const double* n,
                                double* err) {
  const double u = ORC_U32;
  double len = sqrt(n[0] * n[0] + n[1] * n[1]);
  double nx = n[0] / len, ny = n[1] / len;
  orc_face_state S[2];
  double e_p[2], e_c[2], e_un[2], spd[2];
  int k;
  orc_to_face_frame(UL, nx, ny, &S[0]);
  orc_to_face_frame(UR, nx, ny, &S[1]);
  for (k = 0; k < 2; ++k) {
    const orc_face_state* X = &S[k];
    double m2 = X->rho * (X->un * X->un + X->ut * X->ut); /* rho |v|^2 */
    spd[k] = fabs(X->un) + fabs(X->ut);
    /* p = (gamma-1)(E - m2/2): the kinetic part carries 4u, the subtraction u */
    e_p[k] = 2.0 * u * (X->E + m2) + u * X->p;
    /* c = sqrt(gamma p / rho): half the relative error of p/rho, plus rounding */
    e_c[k] = X->c * (0.5 * e_p[k] / X->p + 2.5 * u);
    /* u_n = u hx + v hy: velocities (2u), unit normal (4u), products and sum */
    e_un[k] = 8.0 * u * spd[k];
  }
  double cbar = 0.5 * (S[0].c + S[1].c);
  double pbar = 0.5 * (S[0].p + S[1].p);
  double e_cbar = 0.5 * (e_c[0] + e_c[1]) + u * cbar;
  double r_icb = e_cbar / cbar + u; /* relative error of 1 / c-bar */
  double f[ORC_NF];
  orc_closure_features(UL, UR, n, f);
  err[0] = 4.0 * u * f[0]; /* jump exact or one rounding, mean, reciprocal, product */
  err[1] = (e_un[0] + e_un[1] + u * fabs(S[1].un - S[0].un)) / cbar + f[1] * (r_icb + u);
  err[2] = (e_un[0] + e_un[1] + u * fabs(S[1].ut - S[0].ut)) / cbar + f[2] * (r_icb + u);
  err[3] = (e_p[0] + e_p[1] + u * fabs(S[1].p - S[0].p)) / pbar +
           f[3] * (0.5 * (e_p[0] + e_p[1]) / pbar + 3.0 * u);
  err[4] = 0.5 * (e_un[0] + e_un[1] + u * fabs(S[0].un + S[1].un)) / cbar + f[4] * (r_icb + u);
  err[5] = 0.0;
  for (k = 0; k < 2; ++k) {
    double t = fabs(S[k].un) / S[k].c;
    err[5] += e_un[k] / S[k].c + t * (e_c[k] / S[k].c + 2.0 * u);
  }
  err[5] += u * (fabs(S[0].un) / S[0].c + fabs(S[1].un) / S[1].c);
  err[6] = (S[0].c < S[1].c ? e_c[0] : e_c[1]) / cbar + f[6] * (r_icb + u);
  err[7] = (S[0].c < S[1].c ? e_c[1] : e_c[0]) / cbar + f[7] * (r_icb + u);
  for (k = 0; k < ORC_NF; ++k) err[k] *= ORC_ERR_SAFETY;
}

/* Interval of the scale over every admissible rounding (test support).
 * Each bfloat16 operand is replaced by the interval of bfloat16 values that
 * its admissible FP32 results round to (rounding is monotone, so the ends
 * are the roundings of the ends of the error window); the intervals are
 * carried through the layers in FP64 in centre-radius form (exact weights
 * times an interval), the ReLUs and the sigmoid are monotone and map ends to
 * ends.  The FP32 accumulation of layer 1 is charged 16 * 2^-23 of the sum
 * of the magnitudes of its terms (products of bfloat16 values are exact in
 * FP32; the sum may be rounded or truncated at every addition).
 *   feat_err  nullable: error bounds of the features
 *             (orc_closure_feature_errors); NULL takes the features as exact.
 * Writes [*s_lo, *s_hi] and returns 1 when every rounding is determined (each
 * operand interval is a single bfloat16 value), else 0.  Rounding errors of
 * an FP32 evaluation of layers 2 and 3 are not included. */
int orc_closure_scale_interval(const double* theta, const double* feat, const double* feat_err,
                               double* s_lo, double* s_hi) {
  const double* th = theta;
  double xlo[ORC_NF], xhi[ORC_NF], hlo[ORC_NH], hhi[ORC_NH], glo[ORC_NH], ghi[ORC_NH];
  int i, j, determined = 1;
  for (j = 0; j < ORC_NF; ++j) {
    double w = feat_err ? feat_err[j] : 0.0;
    double lo = feat[j] - w;
    xlo[j] = orc_round_bf16(lo > 0.0 ? lo : 0.0);
    xhi[j] = orc_round_bf16(feat[j] + w);
    if (xlo[j] != xhi[j]) determined = 0;
  }
  for (i = 0; i < ORC_NH; ++i) {
    double c = th[ORC_OFF_B1 + i], r = 0.0, mag = fabs(th[ORC_OFF_B1 + i]);
    for (j = 0; j < ORC_NF; ++j) {
      double wij = th[ORC_OFF_W1 + i * ORC_NF + j];
      c += wij * 0.5 * (xlo[j] + xhi[j]);
      r += fabs(wij) * 0.5 * (xhi[j] - xlo[j]);
      mag += fabs(wij) * xhi[j];
    }
    double w = 16.0 / 8388608.0 * mag;
    double lo = c - r - w, hi = c + r + w;
    hlo[i] = orc_round_bf16(lo > 0.0 ? lo : 0.0);
    hhi[i] = orc_round_bf16(hi > 0.0 ? hi : 0.0);
    if (hlo[i] != hhi[i]) determined = 0;
  }
  for (i = 0; i < ORC_NH; ++i) {
    double c = th[ORC_OFF_B2 + i], r = 0.0;
    for (j = 0; j < ORC_NH; ++j) {
      double wij = th[ORC_OFF_W2 + i * ORC_NH + j];
      c += wij * 0.5 * (hlo[j] + hhi[j]);
      r += fabs(wij) * 0.5 * (hhi[j] - hlo[j]);
    }
    glo[i] = c - r > 0.0 ? c - r : 0.0;
    ghi[i] = c + r > 0.0 ? c + r : 0.0;
  }
  double zc = th[ORC_OFF_B3], zr = 0.0;
  for (i = 0; i < ORC_NH; ++i) {
    zc += th[ORC_OFF_W3 + i] * 0.5 * (glo[i] + ghi[i]);
    zr += fabs(th[ORC_OFF_W3 + i]) * 0.5 * (ghi[i] - glo[i]);
  }
  /* the same expression as orc_mlp_forward: a determined face gives its bits */
  *s_lo = 0.2 + 1.3 * (1.0 / (1.0 + exp(-(zc - zr))));
  *s_hi = 0.2 + 1.3 * (1.0 / (1.0 + exp(-(zc + zr))));
  return determined;
}

/* orc_closure_scale_interval for every face of a mesh with state U (ghost
 * states as in the residual): s_lo[3n], s_hi[3n], determined[3n]. */
void orc_closure_face_intervals(int64_t n, const int32_t* nbr, const double* nrm,
                                const double* uinf, const double* U, const double* theta,
                                double* s_lo, double* s_hi, int32_t* determined) {
  int64_t c;
  int k;
  for (c = 0; c < n; ++c)
    for (k = 0; k < 3; ++k) {
      double UR[4], f[ORC_NF], e[ORC_NF];
      const double* nk = nrm + 6 * c + 2 * k;
      orc_neighbour_state(c, k, nbr, nrm, uinf, U, UR);
      orc_closure_features(U + 4 * c, UR, nk, f);
      orc_closure_feature_errors(U + 4 * c, UR, nk, e);
      determined[3 * c + k] =
          orc_closure_scale_interval(theta, f, e, s_lo + 3 * c + k, s_hi + 3 * c + k);
    }
}

/* ------------------------------------------------------------------------ */
/* Semi-discrete residual dU/dt = -(1/V_T) sum_f F_f . n_f   (Eq. 4)        */
/* ------------------------------------------------------------------------ */

static void orc_neighbour_state(int64_t c, int k, const int32_t* nbr, const double* nrm,
                                const double* uinf, const double* U, double* UR) {
  int32_t m = nbr[3 * c + k];
  if (m >= 0)
    memcpy(UR, U + 4 * (int64_t)m, 4 * sizeof(double));
  else
    orc_ghost(m, U + 4 * c, nrm + 6 * c + 2 * k, uinf, UR);
}

/* theta == NULL: plain Lax-Friedrichs.  scales_out (nullable, n*3) receives
 * the dissipation scale used on each face. */
int orc_residual(int64_t n, const int32_t* nbr, const double* nrm, const double* vol,
                 const double* uinf, const double* U, const double* theta, int32_t bf16_acts,
                 double* R, double* scales_out) {
  int64_t c;
  int k, q;
  for (c = 0; c < n; ++c) {
    double sum[4] = {0.0, 0.0, 0.0, 0.0};
    for (k = 0; k < 3; ++k) {
      double UR[4], F[4];
      const double* nk = nrm + 6 * c + 2 * k;
      orc_neighbour_state(c, k, nbr, nrm, uinf, U, UR);
      double s = theta ? orc_closure_scale(theta, bf16_acts, U + 4 * c, UR, nk) : 1.0;
      if (scales_out) scales_out[3 * c + k] = s;
      orc_face_flux(U + 4 * c, UR, nk, s, F);
      for (q = 0; q < 4; ++q) sum[q] += F[q];
    }
    for (q = 0; q < 4; ++q) R[4 * c + q] = -sum[q] / vol[c];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Time step (reading R1) and conserved totals.                              */
/* ------------------------------------------------------------------------ */

/* 2 V / (P (|v| + c)) for one cell */
double orc_cell_dt_bound(const double* U, const double* nrm_cell, double v) {
  double perim = 0.0;
  int k;
  for (k = 0; k < 3; ++k) {
    double nx = nrm_cell[2 * k], ny = nrm_cell[2 * k + 1];
    perim += sqrt(nx * nx + ny * ny);
  }
  double u = U[1] / U[0], w = U[2] / U[0];
  double lam = sqrt(u * u + w * w) + orc_sound_speed(U[0], orc_pressure(U));
  return 2.0 * v / (perim * lam);
}

double orc_dt(int64_t n, const double* nrm, const double* vol, const double* U, double cfl) {
  if (cfl < 0.0) return -cfl;
  double m = INFINITY;
  int64_t c;
  for (c = 0; c < n; ++c) {
    double b = orc_cell_dt_bound(U + 4 * c, nrm + 6 * c, vol[c]);
    if (b < m) m = b;
  }
  return cfl * m;
}

/* sum_T V_T U_T, the discrete mass, momentum and energy (Eq. 1a-1c) */
void orc_totals(int64_t n, const double* vol, const double* U, double* out) {
  int64_t c;
  int q;
  for (q = 0; q < 4; ++q) out[q] = 0.0;
  for (c = 0; c < n; ++c)
    for (q = 0; q < 4; ++q) out[q] += vol[c] * U[4 * c + q];
}

/* ------------------------------------------------------------------------ */
/* Time loop: forward Euler (Eq. 6 and the update equation of Sec. 6.2.2);  */
/* scheme 1 is the two-stage Heun / SSP-RK2 extension with the same dt.     */
/* Each step's dt is clamped so that the time advanced never passes t_stop  */
/* (t_stop <= 0: no limit); steps with nothing left to advance are skipped. */
/* Returns 0, or 1 if a non-finite state or non-positive density/pressure   */
/* appeared (the state is left as computed).                               */
/* ------------------------------------------------------------------------ */

static int orc_state_bad(int64_t n, const double* U) {
  int64_t c;
  for (c = 0; c < n; ++c) {
    const double* u = U + 4 * c;
    if (!isfinite(u[0]) || !isfinite(u[1]) || !isfinite(u[2]) || !isfinite(u[3])) return 1;
    if (!(u[0] > 0.0) || !(orc_pressure(u) > 0.0)) return 1;
  }
  return 0;
}

int orc_run(int64_t n, const int32_t* nbr, const double* nrm, const double* vol,
            const double* uinf, double* U, int64_t nsteps, double cfl, double t_stop,
            int32_t scheme, const double* theta, int32_t bf16_acts, double* t_out,
            int64_t* steps_out) {
  double* R = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
  double* Us = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
  double t = 0.0;
  int64_t it, i, done = 0;
  int bad = 0;
  if (!R || !Us) {
    free(R);
    free(Us);
    return ORC_E_NOMEM;
  }
  for (it = 0; it < nsteps; ++it) {
    double dt = orc_dt(n, nrm, vol, U, cfl);
    if (t_stop > 0.0) {
      if (t_stop - t < dt) dt = t_stop - t;
      if (!(dt > 0.0)) break;
    }
    orc_residual(n, nbr, nrm, vol, uinf, U, theta, bf16_acts, R, NULL);
    if (scheme == 0) {
      for (i = 0; i < 4 * n; ++i) U[i] = U[i] + dt * R[i];
    } else {
      for (i = 0; i < 4 * n; ++i) Us[i] = U[i] + dt * R[i];
      orc_residual(n, nbr, nrm, vol, uinf, Us, theta, bf16_acts, R, NULL);
      for (i = 0; i < 4 * n; ++i) U[i] = 0.5 * U[i] + 0.5 * (Us[i] + dt * R[i]);
    }
    t += dt;
    ++done;
    if (orc_state_bad(n, U)) {
      bad = 1;
      break;
    }
  }
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = done;
  free(R);
  free(Us);
  return bad;
}

/* ------------------------------------------------------------------------ */
/* One-step training loss of the learned closure and its gradient.          */
/*   U1 = U0 + dt * R(U0; theta)               (forward Euler, fixed dt)     */
/*   L  = sum_T V_T sum_q ((U1 - Ut)_q / w_q)^2                              */
/* The gradient follows the chain  L -> U1 -> F_f -> s_f -> theta, with      */
/* dF_f/ds_f = -1/2 |n| (|u-bar| + c-bar) (U_R - U_L) from Eq. 5.            */
/* ------------------------------------------------------------------------ */

double orc_closure_loss_grad(int64_t n, const int32_t* nbr, const double* nrm, const double* vol,
                             const double* uinf, const double* U0, const double* Ut, double dt,
                             const double* w, const double* theta, int32_t bf16_acts,
                             double* grad) {
  double* R = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
  int64_t c;
  int k, q;
  double loss = 0.0;
  if (!R) return NAN;
  orc_residual(n, nbr, nrm, vol, uinf, U0, theta, bf16_acts, R, NULL);
  if (grad)
    for (q = 0; q < ORC_NPARAM; ++q) grad[q] = 0.0;
  for (c = 0; c < n; ++c) {
    double gU1[4];
    for (q = 0; q < 4; ++q) {
      double d = (U0[4 * c + q] + dt * R[4 * c + q] - Ut[4 * c + q]) / w[q];
      loss += vol[c] * d * d;
      gU1[q] = 2.0 * vol[c] * d / w[q];
    }
    if (!grad) continue;
    for (k = 0; k < 3; ++k) {
      double UR[4], f[ORC_NF];
      const double* UL = U0 + 4 * c;
      const double* nk = nrm + 6 * c + 2 * k;
      orc_mlp_trace tr;
      orc_neighbour_state(c, k, nbr, nrm, uinf, U0, UR);
      orc_closure_features(UL, UR, nk, f);
      orc_mlp_forward(theta, f, bf16_acts, &tr);
      /* d(flux)/d(s): rerun the flux with scale 1 and 0 (it is affine in s) */
      double F1[4], F0[4], gs = 0.0;
      orc_face_flux(UL, UR, nk, 1.0, F1);
      orc_face_flux(UL, UR, nk, 0.0, F0);
      for (q = 0; q < 4; ++q) gs += gU1[q] * (-dt / vol[c]) * (F1[q] - F0[q]);
      orc_mlp_backward(theta, &tr, gs, grad);
    }
  }
  free(R);
  return loss;
}

/* ------------------------------------------------------------------------ */
/* Renumbering diagnostics of Sec. 4.1 on the cell graph, labels = indices.  */
/* ------------------------------------------------------------------------ */

/* B_f(G) = max over edges |f(v) - f(u)| */
int64_t orc_bandwidth(int64_t n, const int32_t* nbr) {
  int64_t c, b = 0;
  int k;
  for (c = 0; c < n; ++c)
    for (k = 0; k < 3; ++k) {
      int32_t m = nbr[3 * c + k];
      if (m >= 0) {
        int64_t d = c > m ? c - m : m - c;
        if (d > b) b = d;
      }
    }
  return b;
}

/* S_BW = max_i E(i) - S(i), with s(i), e(i) the smallest and largest label
 * among the neighbours of the node labelled i, S a suffix minimum of s and E
 * a prefix maximum of e.  Written straight from the definition (quadratic):
 * for every i the two scans run over the whole label range. */
int64_t orc_serial_bandwidth(int64_t n, const int32_t* nbr) {
  int64_t i, j, best = 0;
  int k;
  int64_t* s = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* e = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!s || !e) {
    free(s);
    free(e);
    return -1;
  }
  for (i = 0; i < n; ++i) {
    s[i] = INT64_MAX;
    e[i] = INT64_MIN;
    for (k = 0; k < 3; ++k) {
      int32_t m = nbr[3 * i + k];
      if (m >= 0) {
        if (m < s[i]) s[i] = m;
        if (m > e[i]) e[i] = m;
      }
    }
  }
  for (i = 0; i < n; ++i) {
    int64_t S = INT64_MAX, E = INT64_MIN;
    for (j = i; j < n; ++j)
      if (s[j] < S) S = s[j];
    for (j = 0; j <= i; ++j)
      if (e[j] > E) E = e[j];
    if (S != INT64_MAX && E != INT64_MIN && E - S > best) best = E - S;
  }
  free(s);
  free(e);
  return best;
}
