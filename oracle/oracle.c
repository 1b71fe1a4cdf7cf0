/*
 * oracle.c -- plain, slow, FP64 CPU reference for the unbinned maximum-likelihood
 * path of GooFit (Andreassen et al., "GooFit: A library for massively parallelising
 * maximum-likelihood fits", arXiv:1311.1753).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this
 * file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * legs use it.  It shares no code, header, table or constant generator with the CUDA
 * library under paper_1311_1753_gb300/.
 *
 * What it computes (Sec. 2 and Sec. 4 of the paper: a PDF built from variables and
 * composed PDFs, evaluated per event, a per-event metric summed over events, minimised
 * by MINUIT):
 *
 *   NLL(theta) = - sum_i log P(x_i; theta)
 *
 * with P normalised on the observable ranges.  Every leaf PDF is normalised on its own
 * observable range, sums ("AddPdf", Sec. 3) take fractions of normalised components
 * and products ("ProdPdf", Sec. 3, Listing 2) multiply normalised components of
 * distinct observables.  Sums are compensated (Neumaier) and in fixed event order.
 *
 * Readings where the paper is silent:
 *  - Voigtian = Gaussian (std sigma) convolved with a Breit-Wigner of FWHM Gamma,
 *    V(x) = Re w(z) / (sigma sqrt(2 pi)),  z = (x - mu + i Gamma/2) / (sigma sqrt 2).
 *  - Leaves without a closed-form integral on a finite range (Voigtian, threshold)
 *    are normalised by the midpoint rule on nbins equal bins of the range.
 *  - Threshold background  B(x) = (x-x0)^p exp(-c (x-x0)) for x > x0, else 0.
 *  - Dalitz model (Sec. 4, the D0 -> pi+ pi- pi0 amplitude analysis): coherent sum
 *    A = a_NR + sum_r c_r F_L S_L BW_r with relativistic Breit-Wigners, Blatt-Weisskopf
 *    barrier factors at the resonance vertex and Zemach spin factors; P = |A|^2,
 *    normalised on a cell-centre grid over the kinematic region.
 *
 *  - Later parts, each in its own section below with its reading: binned metrics,
 *    the lattice ConvolutionPdf and the relativistic Breit-Wigner line shape, MappedPdf
 *    and CompositePdf, the time-dependent (mixing) Dalitz model.
 *
 * Pins (tests/test_oracle_pins.py): closed forms, library routines, four-vector
 * kinematics, quadrature and finite differences for every function.  Parity unpinned:
 * the physics conventions of the Dalitz and mixing readings (barrier radius, Zemach
 * factors, the CP-conjugate amplitude, q/p = 1) -- the paper prints no worked number
 * that fixes them, so the oracle and the CUDA path share the reading.
 *
 * Faddeeva function: trapezoidal rule on the integral representation
 *   w(z) = (i/pi) Int e^{-t^2}/(z - t) dt   (Im z > 0)
 * with the residue correction for the pole of the integrand (the method of Matta &
 * Reichel 1971 / Hunter & Regan 1972), derived here by contour integration; see
 * orc_faddeeva.  The CUDA library uses a different method (Weideman 1994).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_SQRTPI 1.77245385090551602730
#define ORC_SQRT2 1.41421356237309504880

/* ------------------------------------------------------------------------------ */
/* Compensated summation (Neumaier): fixed order, used for every sum over events.  */
/* ------------------------------------------------------------------------------ */
typedef struct { double s, c; } orc_acc;
static void acc_add(orc_acc* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double acc_get(const orc_acc* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------------ */
/* Faddeeva function w(z) = exp(-z^2) erfc(-i z), Im z > 0.                        */
/*                                                                                  */
/* Let f(t) = e^{-t^2}/(z - t).  The trapezoidal sum T = h sum_n f(nh) differs from */
/* Int f by the residue of f * pi cot(pi t / h) at t = z plus terms of order        */
/* exp(-pi^2/h^2).  Working the contour integral around the strip |Im t| < pi/h    */
/* gives, for 0 < Im z < pi/h,                                                     */
/*   w(z) = (i h / pi) sum_n e^{-n^2 h^2}/(z - n h) + 2 e^{-z^2}/(1 - e^{-2 pi i z/h}) */
/* and the same without the second term for Im z >= pi/h.  With h = 0.4 the        */
/* neglected terms are ~ e^{-61.7}; |n h| <= 8 keeps every dropped summand below    */
/* e^{-64} of the leading one.                                                      */
/* ------------------------------------------------------------------------------ */
void orc_faddeeva(double x, double y, double* wre, double* wim) {
  const double h = 0.4;
  const int nmax = 20; /* n h <= 8 */
  orc_acc sre = {0, 0}, sim = {0, 0};
  for (int n = -nmax; n <= nmax; ++n) {
    double t = n * h;
    double e = exp(-t * t);
    /* (i h/pi) e / (z - t):  1/(z - t) = (x - t - i y)/((x-t)^2 + y^2) */
    double dx = x - t;
    double den = dx * dx + y * y;
    double inv_re = dx / den, inv_im = -y / den;
    /* multiply by i: (a + ib) i = -b + i a */
    acc_add(&sre, -(h / ORC_PI) * e * inv_im);
    acc_add(&sim, (h / ORC_PI) * e * inv_re);
  }
  double re = acc_get(&sre), im = acc_get(&sim);
  if (y < ORC_PI / h) {
    /* e^{-z^2} = e^{y^2 - x^2} (cos 2xy - i sin 2xy) */
    double mag = exp(y * y - x * x);
    double ez_re = mag * cos(2 * x * y), ez_im = -mag * sin(2 * x * y);
    /* e^{-2 pi i z/h} = e^{2 pi y/h} e^{-i phi}, phi = 2 pi (x - k h)/h with k the nearest
     * node: the phase is taken relative to the same node t_k = k h as the sum above, so
     * the pole of the correction and the pole of the k-th summand cancel consistently. */
    double k = nearbyint(x / h);
    double phi = 2 * ORC_PI * (x - k * h) / h;
    double em = expm1(2 * ORC_PI * y / h);
    double sh = sin(0.5 * phi);
    /* d = 1 - (1 + em) e^{-i phi} = -em cos(phi) + 2 sin^2(phi/2) + i (1 + em) sin(phi) */
    double d_re = -em * cos(phi) + 2 * sh * sh;
    double d_im = (1 + em) * sin(phi);
    double dd = d_re * d_re + d_im * d_im;
    /* 2 ez / d */
    double q_re = 2 * (ez_re * d_re + ez_im * d_im) / dd;
    double q_im = 2 * (ez_im * d_re - ez_re * d_im) / dd;
    re += q_re;
    im += q_im;
  }
  *wre = re;
  *wim = im;
}

/* w'(z) = -2 z w(z) + 2 i / sqrt(pi)  (differentiate e^{-z^2} erfc(-iz)). */
static void faddeeva_deriv(double x, double y, double wre, double wim, double* dre, double* dim) {
  *dre = -2 * (x * wre - y * wim);
  *dim = -2 * (x * wim + y * wre) + 2 / ORC_SQRTPI;
}

/* ------------------------------------------------------------------------------ */
/* 1D model: a tree of leaves and combinators (Sec. 3).                            */
/* ------------------------------------------------------------------------------ */
enum {
  ORC_EXP = 1,    /* e^{alpha x}                         par: alpha          (Listing 1) */
  ORC_GAUSS = 2,  /* exp(-(x-mu)^2 / (2 sigma^2))        par: mu, sigma      (Listing 3) */
  ORC_VOIGT = 3,  /* Re w(z)/(sigma sqrt(2 pi))          par: mu, sigma, Gamma           */
  ORC_THRESH = 4, /* (x-x0)^p e^{-c (x-x0)}, x > x0      par: x0, p, c                   */
  ORC_POLY = 5,   /* sum_k a_k x^k                       par: a_0 .. a_deg               */
  ORC_RELBW = 6,  /* relativistic Breit-Wigner line shape (Sec. 4, the D*+ width fit):
                   * m Gamma(m) / ((m0^2 - m^2)^2 + m0^2 Gamma(m)^2), m = x + shift,
                   * m0 = dm0 + shift, Gamma(m) = Gamma0 (q/q0)^{2L+1} (m0/m) F_L^2,
                   * zero at or below threshold m <= ma + mb;
                   *                                     par: dm0, Gamma0, shift, ma, mb, R;
                   *                                     aux: L (orbital angular momentum) */
  ORC_ADD = 10,   /* sum_k f_k P_k + (1 - sum f) P_last  par: f_0 .. f_{n-2}  (AddPdf)   */
  ORC_PROD = 11,  /* prod_k P_k (distinct observables)                        (ProdPdf)  */
  ORC_CONV = 12,  /* ConvolutionPdf (Sec. 3): model (child 0, observable obs) convolved
                   * with a resolution (child 1, over its own residual observable), on a
                   * lattice of aux bins of obs's range; see conv_table              */
  ORC_MAPPED = 13,   /* MappedPdf (Sec. 3): child k on [b_{k-1}, b_k) of obs's range
                      * (b_{-1} = lo, b_{n-1} = hi; par: the n-1 interior boundaries),
                      * each child normalised on the whole range, the result normalised
                      * by the midpoint rule on nbins bins                              */
  ORC_COMPOSITE = 14 /* CompositePdf (Sec. 3): f(g(x)) with g the core leaf (child 0, its
                      * unnormalised shape over obs) and f the shell leaf (child 1:
                      * exponential, Gaussian or polynomial, unnormalised shape of the
                      * core's value), normalised by the midpoint rule on nbins bins     */
};

#define ORC_MAXPAR 16
#define ORC_MAXCHILD 8
typedef struct {
  int32_t type;
  int32_t obs;
  int32_t npar;
  int32_t par[ORC_MAXPAR];
  int32_t nchild;
  int32_t child[ORC_MAXCHILD];
  int32_t aux; /* RELBW: L; CONV: lattice bins */
} orc_node;

typedef struct {
  int32_t nnodes;
  int32_t root;
  const orc_node* nodes;
  int32_t nobs;
  const double* lo;
  const double* hi;
  int32_t nbins; /* midpoint-rule bins for grid-normalised leaves */
  int32_t ndata; /* data columns: observables 0 .. ndata-1 (the rest are residual
                    observables of resolution functions) */
} orc_model;

/* Per-evaluation state: normalisation of every node and its gradient, and the lattice
 * table of every convolution node ((1 + np) x (L + 1): C_i, then dC_i/dp_k). */
typedef struct {
  double* N;
  double* dN;
  double** tab;
} orc_state;

/* Relativistic Breit-Wigner line shape (ORC_RELBW).  With s = m^2 and the squared
 * break-up momentum of a, b at s, q^2(s) = (s - (ma+mb)^2)(s - (ma-mb)^2)/(4 s),
 * Blatt-Weisskopf B_L(z) = 1, 1 + z, 9 + 3z + z^2 (z = q^2 R^2), F_L^2 = B_L(z0)/B_L(z),
 *   Gamma(m) = Gamma0 (q/q0)^{2L+1} (m0/m) F_L^2,   f = m Gamma / D,
 *   D = (m0^2 - m^2)^2 + m0^2 Gamma^2.
 * Derivatives (m0 enters through q0, z0, m0/m and D):
 *   dGamma/dGamma0 = Gamma/Gamma0,
 *   dln Gamma/dm0 = -(2L+1) dln q0/dm0 + 1/m0 + B_L'(z0)/B_L(z0) dz0/dm0,
 *   dq0^2/dm0 = 2 m0 (s0^2 - A B)/(4 s0^2), A = (ma+mb)^2, B = (ma-mb)^2, s0 = m0^2,
 *   df = m dGamma/D - f dD/D,  dD = 4 m0 (m0^2 - m^2) dm0 + 2 m0 Gamma^2 dm0
 *                                   + 2 m0^2 Gamma dGamma. */
static double rb_poly(int L, double z) { return L == 0 ? 1.0 : L == 1 ? 1.0 + z : 9.0 + 3.0 * z + z * z; }
static double rb_poly_dz(int L, double z) { return L == 0 ? 0.0 : L == 1 ? 1.0 : 3.0 + 2.0 * z; }
static double relbw_shape(const orc_node* nd, const double* p, double x, double* dr) {
  double dm0 = p[nd->par[0]], g0 = p[nd->par[1]], shift = p[nd->par[2]];
  double ma = p[nd->par[3]], mb = p[nd->par[4]], R = p[nd->par[5]];
  int L = nd->aux;
  double m = x + shift, m0 = dm0 + shift;
  /* distances to threshold from the observable directly: s - A = (m - ma - mb)(m + ma + mb)
   * with m - ma - mb = x - (ma + mb - shift), free of the cancellation of s - A near
   * threshold */
  double thr = ma + mb - shift;
  if (dr) for (int k = 0; k < 6; ++k) dr[k] = 0.0;
  if (!(x - thr > 0)) return 0.0;
  double A = (ma + mb) * (ma + mb), B = (ma - mb) * (ma - mb);
  double s = m * m, s0 = m0 * m0;
  double q2 = (x - thr) * (m + ma + mb) * (s - B) / (4 * s);
  double q02 = (dm0 - thr) * (m0 + ma + mb) * (s0 - B) / (4 * s0);
  double z = q2 * R * R, z0 = q02 * R * R;
  double F2 = rb_poly(L, z0) / rb_poly(L, z);
  double G = g0 * pow(q2 / q02, L + 0.5) * (m0 / m) * F2;
  /* m0^2 - m^2 = (dm0 - x)(m0 + m): no cancellation near the pole */
  double ds = (dm0 - x) * (m0 + m);
  double D = ds * ds + s0 * G * G;
  double f = m * G / D;
  if (dr) {
    /* Gamma0 */
    double dG = G / g0;
    double dD = 2 * s0 * G * dG;
    dr[1] = m * dG / D - f * dD / D;
    /* dm0 */
    double dq02 = 2 * m0 * (s0 * s0 - A * B) / (4 * s0 * s0);
    double dlnG = -(L + 0.5) * dq02 / q02 + 1.0 / m0 + rb_poly_dz(L, z0) * R * R * dq02 / rb_poly(L, z0);
    dG = G * dlnG;
    dD = 4 * m0 * ds + 2 * m0 * G * G + 2 * s0 * G * dG;
    dr[0] = m * dG / D - f * dD / D;
  }
  return f;
}

/* Unnormalised leaf shape r(x) and its partial derivatives with respect to the
 * leaf's own parameters (dr[k] for par[k]).  RELBW: derivatives for dm0 and Gamma0
 * only (its other parameters are constants of the decay). */
static double leaf_shape(const orc_node* nd, const double* p, double x, double* dr) {
  switch (nd->type) {
    case ORC_RELBW:
      return relbw_shape(nd, p, x, dr);
    case ORC_EXP: {
      double a = p[nd->par[0]];
      double v = exp(a * x);
      if (dr) dr[0] = x * v;
      return v;
    }
    case ORC_GAUSS: {
      double mu = p[nd->par[0]], s = p[nd->par[1]];
      double u = (x - mu) / s;
      double v = exp(-0.5 * u * u);
      if (dr) {
        dr[0] = v * u / s;
        dr[1] = v * u * u / s;
      }
      return v;
    }
    case ORC_VOIGT: {
      double mu = p[nd->par[0]], s = p[nd->par[1]], G = p[nd->par[2]];
      double zr = (x - mu) / (s * ORC_SQRT2), zi = G / (2 * s * ORC_SQRT2);
      double wre, wim;
      orc_faddeeva(zr, zi, &wre, &wim);
      double pref = 1.0 / (s * sqrt(2 * ORC_PI));
      double v = wre * pref;
      if (dr) {
        double dre, dim;
        faddeeva_deriv(zr, zi, wre, wim, &dre, &dim);
        /* dz/dmu = -1/(s sqrt2);  dz/dGamma = i/(2 s sqrt2);  dz/ds = -z/s */
        dr[0] = pref * (-dre / (s * ORC_SQRT2));
        dr[2] = pref * (-dim / (2 * s * ORC_SQRT2));
        /* Re(w' * (-z/s)) = -(dre zr - dim zi)/s */
        dr[1] = pref * (-(dre * zr - dim * zi) / s) - v / s;
      }
      return v;
    }
    case ORC_THRESH: {
      double x0 = p[nd->par[0]], pw = p[nd->par[1]], c = p[nd->par[2]];
      double t = x - x0;
      if (!(t > 0)) {
        if (dr) dr[0] = dr[1] = dr[2] = 0;
        return 0.0;
      }
      double v = pow(t, pw) * exp(-c * t);
      if (dr) {
        dr[0] = v * (c - pw / t);
        dr[1] = v * log(t);
        dr[2] = -t * v;
      }
      return v;
    }
    case ORC_POLY: {
      double v = 0, xk = 1;
      for (int k = 0; k < nd->npar; ++k) {
        v += p[nd->par[k]] * xk;
        if (dr) dr[k] = xk;
        xk *= x;
      }
      return v;
    }
  }
  return NAN;
}

/* d f/d u of an analytic shell shape f(u) (exponential, Gaussian, polynomial). */
static double shell_du(const orc_node* nd, const double* p, double u) {
  if (nd->type == ORC_EXP) return p[nd->par[0]] * exp(p[nd->par[0]] * u);
  if (nd->type == ORC_GAUSS) {
    double mu = p[nd->par[0]], s = p[nd->par[1]], t = (u - mu) / s;
    return -t / s * exp(-0.5 * t * t);
  }
  double d = 0, uk = 1; /* polynomial: sum_k k a_k u^{k-1} */
  for (int k = 1; k < nd->npar; ++k) {
    d += k * p[nd->par[k]] * uk;
    uk *= u;
  }
  return d;
}

static int is_leaf(int type) { return type >= ORC_EXP && type <= ORC_RELBW; }
static int grid_normalised(int type) {
  return type == ORC_VOIGT || type == ORC_THRESH || type == ORC_RELBW;
}

/* Integral of e^{a x} on [lo, hi] and its a-derivative (Int x e^{a x}). */
static void exp_integral(double a, double lo, double hi, double* N, double* dN) {
  double m = fmax(fabs(lo), fabs(hi));
  if (fabs(a) * m < 0.1) {
    /* Taylor series of the integrand in a, integrated term by term (the closed form
     * below cancels to ~|a m|^-1 ulps when |a| m is small). */
    double n = 0, d = 0, ak = 1, fact = 1;
    for (int k = 0; k <= 24; ++k) {
      if (k > 0) { ak *= a; fact *= k; }
      n += ak / fact * (pow(hi, k + 1) - pow(lo, k + 1)) / (k + 1);
      d += ak / fact * (pow(hi, k + 2) - pow(lo, k + 2)) / (k + 2);
    }
    *N = n;
    *dN = d;
    return;
  }
  double eh = exp(a * hi), el = exp(a * lo);
  *N = (eh - el) / a;
  *dN = (hi * eh - lo * el) / a - *N / a;
}

/* Gaussian integral on [lo, hi] via erfc differences that avoid cancellation in the
 * tails, and its derivatives in mu and sigma. */
static void gauss_integral(double mu, double s, double lo, double hi, double* N, double* dmu, double* ds) {
  double a = (lo - mu) / s, b = (hi - mu) / s;
  double diff; /* Phi(b) - Phi(a) */
  if (a >= 0) diff = 0.5 * (erfc(a / ORC_SQRT2) - erfc(b / ORC_SQRT2));
  else if (b <= 0) diff = 0.5 * (erfc(-b / ORC_SQRT2) - erfc(-a / ORC_SQRT2));
  else diff = 1.0 - 0.5 * erfc(-a / ORC_SQRT2) - 0.5 * erfc(b / ORC_SQRT2);
  *N = s * sqrt(2 * ORC_PI) * diff;
  double ea = exp(-0.5 * a * a), eb = exp(-0.5 * b * b);
  *dmu = ea - eb;
  *ds = a * ea - b * eb + *N / s;
}

/* Normalisation integral of every leaf over its observable range, and its
 * gradient with respect to all parameters (dN[node * np + k]).  Non-leaves get 1. */
int orc_norms(const orc_model* m, const double* p, int np, double* N, double* dN) {
  memset(dN, 0, sizeof(double) * (size_t)m->nnodes * np);
  for (int i = 0; i < m->nnodes; ++i) {
    const orc_node* nd = &m->nodes[i];
    N[i] = 1.0;
    if (!is_leaf(nd->type)) continue;
    double lo = m->lo[nd->obs], hi = m->hi[nd->obs];
    double* g = dN + (size_t)i * np;
    if (nd->type == ORC_EXP) {
      double n, d;
      exp_integral(p[nd->par[0]], lo, hi, &n, &d);
      N[i] = n;
      g[nd->par[0]] += d;
    } else if (nd->type == ORC_GAUSS) {
      double n, dmu, ds;
      gauss_integral(p[nd->par[0]], p[nd->par[1]], lo, hi, &n, &dmu, &ds);
      N[i] = n;
      g[nd->par[0]] += dmu;
      g[nd->par[1]] += ds;
    } else if (nd->type == ORC_POLY) {
      double n = 0;
      for (int k = 0; k < nd->npar; ++k) {
        double ik = (pow(hi, k + 1) - pow(lo, k + 1)) / (k + 1);
        n += p[nd->par[k]] * ik;
        g[nd->par[k]] += ik;
      }
      N[i] = n;
    } else if (grid_normalised(nd->type)) {
      /* Midpoint rule: N = h sum_b r(lo + (b + 1/2) h). */
      double h = (hi - lo) / m->nbins;
      orc_acc s = {0, 0};
      orc_acc ds[ORC_MAXPAR];
      memset(ds, 0, sizeof(ds));
      double dr[ORC_MAXPAR];
      for (int b = 0; b < m->nbins; ++b) {
        double x = lo + (b + 0.5) * h;
        acc_add(&s, leaf_shape(nd, p, x, dr));
        for (int k = 0; k < nd->npar; ++k) acc_add(&ds[k], dr[k]);
      }
      N[i] = h * acc_get(&s);
      for (int k = 0; k < nd->npar; ++k) g[nd->par[k]] += h * acc_get(&ds[k]);
    } else {
      return -1;
    }
  }
  return 0;
}

static double node_value(const orc_model* m, int i, const double* p, int np,
                         const orc_state* st, const double* x, double* g);

/* MappedPdf / CompositePdf before their normalisation, with the gradient g[np]:
 *  mapped:    P_k(x) for the interval k holding x (the last interval is closed);
 *  composite: f(u), u = g(x) (both unnormalised leaf shapes), d/dtheta = df/dtheta_f +
 *             f'(u) du/dtheta_g. */
static double mapped_raw(const orc_model* m, int i, const double* p, int np,
                         const orc_state* st, const double* x, double* g) {
  const orc_node* nd = &m->nodes[i];
  double xv = x[nd->obs];
  if (nd->type == ORC_MAPPED) {
    int k = 0;
    while (k < nd->nchild - 1 && xv >= p[nd->par[k]]) ++k;
    return node_value(m, nd->child[k], p, np, st, x, g);
  }
  const orc_node* core = &m->nodes[nd->child[0]];
  const orc_node* shell = &m->nodes[nd->child[1]];
  double dc[ORC_MAXPAR], ds[ORC_MAXPAR];
  double u = leaf_shape(core, p, xv, g ? dc : NULL);
  double f = leaf_shape(shell, p, u, g ? ds : NULL);
  if (g) {
    memset(g, 0, sizeof(double) * np);
    double fu = shell_du(shell, p, u);
    for (int k = 0; k < core->npar; ++k) g[core->par[k]] += fu * dc[k];
    for (int k = 0; k < shell->npar; ++k) g[shell->par[k]] += ds[k];
  }
  return f;
}

/* Normalised value of a node at one event, optionally with its gradient g[np]. */
static double node_value(const orc_model* m, int i, const double* p, int np,
                         const orc_state* st, const double* x, double* g) {
  const orc_node* nd = &m->nodes[i];
  const double* N = st->N;
  const double* dN = st->dN;
  if (is_leaf(nd->type)) {
    double dr[ORC_MAXPAR];
    double r = leaf_shape(nd, p, x[nd->obs], g ? dr : NULL);
    double v = r / N[i];
    if (g) {
      /* d(r/N) = (dr - v dN)/N */
      for (int k = 0; k < np; ++k) g[k] = -v * dN[(size_t)i * np + k] / N[i];
      for (int k = 0; k < nd->npar; ++k) g[nd->par[k]] += dr[k] / N[i];
    }
    return v;
  }
  if (nd->type == ORC_MAPPED || nd->type == ORC_COMPOSITE) {
    /* unnormalised value (mapped_raw), divided by the grid normalisation */
    double v = mapped_raw(m, i, p, np, st, x, g) / N[i];
    if (g)
      for (int q = 0; q < np; ++q) g[q] = g[q] / N[i] - v * dN[(size_t)i * np + q] / N[i];
    return v;
  }
  if (nd->type == ORC_CONV) {
    /* linear interpolation of the lattice table, divided by the node's normalisation */
    const double* T = st->tab[i];
    int L = nd->aux;
    double lo = m->lo[nd->obs], hi = m->hi[nd->obs], h = (hi - lo) / L;
    double sx = (x[nd->obs] - lo) / h;
    int k = (int)floor(sx);
    if (k < 0) k = 0;
    if (k > L - 1) k = L - 1;
    double u = sx - k;
    double c = (1 - u) * T[k] + u * T[k + 1];
    double v = c / N[i];
    if (g)
      for (int q = 0; q < np; ++q) {
        const double* Tq = T + (size_t)(1 + q) * (L + 1);
        g[q] = ((1 - u) * Tq[k] + u * Tq[k + 1]) / N[i] - v * dN[(size_t)i * np + q] / N[i];
      }
    return v;
  }
  if (nd->type == ORC_ADD) {
    int nc = nd->nchild;
    double fsum = 0, v = 0, vlast;
    double* gc = g ? (double*)malloc(sizeof(double) * np) : NULL;
    if (g) memset(g, 0, sizeof(double) * np);
    vlast = node_value(m, nd->child[nc - 1], p, np, st, x, gc);
    for (int k = 0; k < nc - 1; ++k) fsum += p[nd->par[k]];
    v = (1.0 - fsum) * vlast;
    if (g) for (int j = 0; j < np; ++j) g[j] += (1.0 - fsum) * gc[j];
    for (int k = 0; k < nc - 1; ++k) {
      double f = p[nd->par[k]];
      double vk = node_value(m, nd->child[k], p, np, st, x, gc);
      v += f * vk;
      if (g) {
        for (int j = 0; j < np; ++j) g[j] += f * gc[j];
        g[nd->par[k]] += vk - vlast;
      }
    }
    free(gc);
    return v;
  }
  if (nd->type == ORC_PROD) {
    int nc = nd->nchild;
    double vals[ORC_MAXCHILD];
    double* gcs = g ? (double*)malloc(sizeof(double) * np * nc) : NULL;
    double v = 1;
    for (int k = 0; k < nc; ++k) {
      vals[k] = node_value(m, nd->child[k], p, np, st, x, g ? gcs + (size_t)k * np : NULL);
      v *= vals[k];
    }
    if (g) {
      memset(g, 0, sizeof(double) * np);
      for (int k = 0; k < nc; ++k) {
        double others = 1;
        for (int j = 0; j < nc; ++j) if (j != k) others *= vals[j];
        for (int j = 0; j < np; ++j) g[j] += others * gcs[(size_t)k * np + j];
      }
    }
    free(gcs);
    return v;
  }
  return NAN;
}

/* log of the normalised value.  Exponential and Gaussian leaves and products are
 * taken in the log domain (log e^{a x}/N = a x - log N), which is the same quantity
 * without the round trip through exp. */
static double node_logvalue(const orc_model* m, int i, const double* p, int np,
                            const orc_state* st, const double* x, double* g) {
  const orc_node* nd = &m->nodes[i];
  const double* N = st->N;
  const double* dN = st->dN;
  if (nd->type == ORC_EXP) {
    double a = p[nd->par[0]], xv = x[nd->obs];
    if (g) {
      for (int k = 0; k < np; ++k) g[k] = -dN[(size_t)i * np + k] / N[i];
      g[nd->par[0]] += xv;
    }
    return a * xv - log(N[i]);
  }
  if (nd->type == ORC_GAUSS) {
    double mu = p[nd->par[0]], s = p[nd->par[1]], u = (x[nd->obs] - mu) / s;
    if (g) {
      for (int k = 0; k < np; ++k) g[k] = -dN[(size_t)i * np + k] / N[i];
      g[nd->par[0]] += u / s;
      g[nd->par[1]] += u * u / s;
    }
    return -0.5 * u * u - log(N[i]);
  }
  if (nd->type == ORC_PROD) {
    double v = 0;
    double* gc = g ? (double*)malloc(sizeof(double) * np) : NULL;
    if (g) memset(g, 0, sizeof(double) * np);
    for (int k = 0; k < nd->nchild; ++k) {
      v += node_logvalue(m, nd->child[k], p, np, st, x, gc);
      if (g) for (int j = 0; j < np; ++j) g[j] += gc[j];
    }
    free(gc);
    return v;
  }
  double v = node_value(m, i, p, np, st, x, g);
  if (g) for (int j = 0; j < np; ++j) g[j] /= v;
  return log(v);
}

/* ------------------------------------------------------------------------------ */
/* ConvolutionPdf (Sec. 3; Sec. 4: a Breit-Wigner convolved with a resolution of    */
/* several Gaussians).  The paper names the class, not its numerics; the reading    */
/* used here:                                                                      */
/*  - lattice x_i = lo + i h, i = 0..L, h = (hi - lo)/L on the observable's range;  */
/*  - resolution R (normalised on its residual observable's range [rlo, rhi]) at    */
/*    the offsets u_k = k h inside that range, k = kmin..kmax;                     */
/*  - model M (normalised on [lo, hi], evaluated wherever needed) at t = x_i - u_k;  */
/*  - C_i = h sum_k R(u_k) M(x_i - u_k)   (Riemann sum of Int M(t) R(x - t) dt);     */
/*  - C(x) linear between lattice points, P(x) = C(x)/N with N = Int_lo^hi C, the    */
/*    trapezoid sum h (C_0/2 + C_1 + ... + C_{L-1} + C_L/2), exact for the           */
/*    interpolant;                                                                 */
/*  - gradients by differentiating every step.                                     */
/* ------------------------------------------------------------------------------ */
static int subtree_obs(const orc_model* m, int i) {
  const orc_node* nd = &m->nodes[i];
  if (is_leaf(nd->type)) return nd->obs;
  return nd->nchild > 0 ? subtree_obs(m, nd->child[0]) : -1;
}

static int conv_table(const orc_model* m, int i, const double* p, int np, orc_state* st) {
  const orc_node* nd = &m->nodes[i];
  int L = nd->aux, M = nd->child[0], R = nd->child[1];
  int ro = subtree_obs(m, R);
  if (L < 1 || ro < 0 || ro == nd->obs) return -1;
  double lo = m->lo[nd->obs], hi = m->hi[nd->obs], h = (hi - lo) / L;
  int kmin = (int)ceil(m->lo[ro] / h - 1e-9), kmax = (int)floor(m->hi[ro] / h + 1e-9);
  if (kmax < kmin) return -1;
  int J = L + kmax - kmin + 1, K = kmax - kmin + 1;
  double* mt = (double*)calloc((size_t)(1 + np) * J, sizeof(double));
  double* rt = (double*)calloc((size_t)(1 + np) * K, sizeof(double));
  double* T = (double*)calloc((size_t)(1 + np) * (L + 1), sizeof(double));
  double* g = (double*)malloc(sizeof(double) * np);
  double x[16] = {0};
  for (int j = 0; j < J; ++j) {
    x[nd->obs] = lo + (j - kmax) * h;
    mt[j] = node_value(m, M, p, np, st, x, g);
    for (int q = 0; q < np; ++q) mt[(size_t)(1 + q) * J + j] = g[q];
  }
  for (int k = 0; k < K; ++k) {
    x[ro] = (kmin + k) * h;
    rt[k] = node_value(m, R, p, np, st, x, g);
    for (int q = 0; q < np; ++q) rt[(size_t)(1 + q) * K + k] = g[q];
  }
  orc_acc nsum = {0, 0};
  orc_acc* dsum = (orc_acc*)calloc(np, sizeof(orc_acc));
  for (int ii = 0; ii <= L; ++ii) {
    double wt = (ii == 0 || ii == L) ? 0.5 : 1.0;
    /* u_k = (kmin + k) h pairs with t = x_ii - u_k, model index j = ii - kmin - k + kmax */
    orc_acc c = {0, 0};
    for (int k = 0; k < K; ++k) acc_add(&c, rt[k] * mt[ii - kmin - k + kmax]);
    T[ii] = h * acc_get(&c);
    acc_add(&nsum, wt * T[ii]);
    for (int q = 0; q < np; ++q) {
      orc_acc d = {0, 0};
      const double* mq = mt + (size_t)(1 + q) * J;
      const double* rq = rt + (size_t)(1 + q) * K;
      for (int k = 0; k < K; ++k) {
        int j = ii - kmin - k + kmax;
        acc_add(&d, rq[k] * mt[j]);
        acc_add(&d, rt[k] * mq[j]);
      }
      T[(size_t)(1 + q) * (L + 1) + ii] = h * acc_get(&d);
      acc_add(&dsum[q], wt * T[(size_t)(1 + q) * (L + 1) + ii]);
    }
  }
  st->N[i] = h * acc_get(&nsum);
  for (int q = 0; q < np; ++q) st->dN[(size_t)i * np + q] = h * acc_get(&dsum[q]);
  st->tab[i] = T;
  free(mt); free(rt); free(g); free(dsum);
  return 0;
}

static void state_free(const orc_model* m, orc_state* st) {
  if (st->tab)
    for (int i = 0; i < m->nnodes; ++i) free(st->tab[i]);
  free(st->tab);
  free(st->N);
  free(st->dN);
}

/* Normalisations of every leaf, then the lattice table and normalisation of every
 * convolution node (their subtrees hold no convolution). */
static int state_init(const orc_model* m, const double* p, int np, orc_state* st) {
  st->N = (double*)malloc(sizeof(double) * m->nnodes);
  st->dN = (double*)malloc(sizeof(double) * m->nnodes * (size_t)(np > 0 ? np : 1));
  st->tab = (double**)calloc(m->nnodes, sizeof(double*));
  if (orc_norms(m, p, np, st->N, st->dN)) { state_free(m, st); return -1; }
  for (int i = 0; i < m->nnodes; ++i)
    if (m->nodes[i].type == ORC_CONV && conv_table(m, i, p, np, st)) { state_free(m, st); return -1; }
  /* MappedPdf / CompositePdf: midpoint rule over their observable's range */
  for (int i = 0; i < m->nnodes; ++i) {
    const orc_node* nd = &m->nodes[i];
    if (nd->type != ORC_MAPPED && nd->type != ORC_COMPOSITE) continue;
    double lo = m->lo[nd->obs], hi = m->hi[nd->obs], h = (hi - lo) / m->nbins;
    double x[16] = {0};
    double* g = (double*)malloc(sizeof(double) * (np > 0 ? np : 1));
    orc_acc s = {0, 0};
    orc_acc* ds = (orc_acc*)calloc(np > 0 ? np : 1, sizeof(orc_acc));
    for (int b = 0; b < m->nbins; ++b) {
      x[nd->obs] = lo + (b + 0.5) * h;
      acc_add(&s, mapped_raw(m, i, p, np, st, x, g));
      for (int q = 0; q < np; ++q) acc_add(&ds[q], g[q]);
    }
    st->N[i] = h * acc_get(&s);
    for (int q = 0; q < np; ++q) st->dN[(size_t)i * np + q] = h * acc_get(&ds[q]);
    free(g);
    free(ds);
  }
  return 0;
}

/* Per-event log P (normalised).  cols[o] is the column of observable o. */
int orc_logpdf(const orc_model* m, const double* p, int np, int64_t n, const double* const* cols,
               double* out) {
  orc_state S, *st = &S;
  if (state_init(m, p, np, st)) return -1;
  double x[16] = {0};
  for (int64_t i = 0; i < n; ++i) {
    for (int o = 0; o < m->ndata; ++o) x[o] = cols[o][i];
    out[i] = node_logvalue(m, m->root, p, np, st, x, NULL);
  }
  state_free(m, st);
  return 0;
}

/* NLL = -sum_i log P_i and, if grad != NULL, its gradient over all np parameters. */
int orc_nll(const orc_model* m, const double* p, int np, int64_t n, const double* const* cols,
            double* nll, double* grad) {
  orc_state S, *st = &S;
  if (state_init(m, p, np, st)) return -1;
  orc_acc s = {0, 0};
  orc_acc* gs = (orc_acc*)calloc(np, sizeof(orc_acc));
  double* g = (double*)malloc(sizeof(double) * np);
  double x[16] = {0};
  for (int64_t i = 0; i < n; ++i) {
    for (int o = 0; o < m->ndata; ++o) x[o] = cols[o][i];
    double lp = node_logvalue(m, m->root, p, np, st, x, grad ? g : NULL);
    acc_add(&s, -lp);
    if (grad) for (int k = 0; k < np; ++k) acc_add(&gs[k], -g[k]);
  }
  *nll = acc_get(&s);
  if (grad) for (int k = 0; k < np; ++k) grad[k] = acc_get(&gs[k]);
  state_free(m, st);
  free(gs); free(g);
  return 0;
}

/* ------------------------------------------------------------------------------ */
/* Binned metrics (Sec. 2: "evaluate" gives the normalised PDF at a point and the   */
/* fit's "metric" turns those values into the quantity minimised, so one PDF serves */
/* maximum-likelihood and chi-squared fits; Sec. 4: the binned D*+ width fit).      */
/* Bin b has centre x_b (one column per observable) and content n_b; its expected   */
/* content is nu_b = K P(x_b), K = (total content) x (bin volume), given by the     */
/* caller.                                                                          */
/*   metric 0:  -sum_b n_b log P(x_b)                 (multinomial likelihood)      */
/*   metric 1:   sum_b (nu_b - n_b log nu_b)          (Poisson likelihood without   */
/*                                                     the constant log n_b!)       */
/*   metric 2:   sum_b (n_b - nu_b)^2 / s2_b          (chi-squared, s2_b the        */
/*                                                     variance of bin b)           */
/* Gradient: d/dtheta = sum_b (d term_b / d P_b) dP_b/dtheta with d term/d P =      */
/* -n_b/P_b, K - n_b/P_b and -2 (n_b - nu_b) K / s2_b respectively (a bin with       */
/* n_b = 0 contributes nothing to metric 0 and K dP_b/dtheta to metric 1; at P_b = 0 */
/* the chi-squared term still moves with nu_b, so the chain goes through P, not      */
/* log P).                                                                          */
/* ------------------------------------------------------------------------------ */
int orc_binned(const orc_model* m, const double* p, int np, int64_t nb, const double* const* cols,
               const double* cnt, const double* s2, double K, int metric, double* val,
               double* grad) {
  if (metric < 0 || metric > 2 || (metric == 2 && !s2)) return -1;
  orc_state S, *st = &S;
  if (state_init(m, p, np, st)) return -1;
  orc_acc s = {0, 0};
  orc_acc* gs = (orc_acc*)calloc(np, sizeof(orc_acc));
  double* g = (double*)malloc(sizeof(double) * np);
  double x[16] = {0};
  for (int64_t b = 0; b < nb; ++b) {
    for (int o = 0; o < m->ndata; ++o) x[o] = cols[o][b];
    double v = node_value(m, m->root, p, np, st, x, grad ? g : NULL); /* P_b, dP_b */
    double lp = log(v);
    double n = cnt[b], term, c;
    if (metric == 0) {
      term = n == 0 ? 0.0 : -n * lp;
      c = n == 0 ? 0.0 : -n / v;
    } else {
      double nu = K * v;
      if (metric == 1) {
        term = n == 0 ? nu : nu - n * (lp + log(K));
        c = n == 0 ? K : K - n / v;
      } else {
        double r = n - nu;
        term = r * r / s2[b];
        c = -2.0 * r * K / s2[b];
      }
    }
    acc_add(&s, term);
    if (grad && c != 0.0) for (int k = 0; k < np; ++k) acc_add(&gs[k], c * g[k]);
  }
  *val = acc_get(&s);
  if (grad) for (int k = 0; k < np; ++k) grad[k] = acc_get(&gs[k]);
  state_free(m, st);
  free(gs); free(g);
  return 0;
}

/* Unnormalised shape of one leaf (for pins against closed forms). */
double orc_leaf_shape(const orc_node* nd, const double* p, double x) {
  return leaf_shape(nd, p, x, NULL);
}

/* ------------------------------------------------------------------------------ */
/* Three-body Dalitz amplitude model (Sec. 4: D0 -> pi+ pi- pi0 with 16 complex     */
/* amplitudes).  Observables s12 = m12^2, s13 = m13^2; s23 follows from             */
/* s12 + s13 + s23 = M^2 + m1^2 + m2^2 + m3^2.                                      */
/* ------------------------------------------------------------------------------ */
typedef struct {
  double M, m1, m2, m3; /* parent and daughter masses (GeV) */
  double R;             /* Blatt-Weisskopf radius (GeV^-1) */
} orc_dkin;

typedef struct {
  int32_t channel; /* 0: (12) with bachelor 3; 1: (13) with bachelor 2; 2: (23) with bachelor 1 */
  int32_t spin;    /* 0, 1, 2 */
  int32_t p_m0, p_g0, p_re, p_im; /* parameter indices */
} orc_res;

/* Kinematic region for a given s12: s23 lies between the values reached when the
 * momenta of particles 2 and 3, in the rest frame of the (12) system, are parallel or
 * antiparallel.  Returns 1 inside, 0 outside. */
int orc_dalitz_inside(const orc_dkin* k, double s12, double s13) {
  double M = k->M, m1 = k->m1, m2 = k->m2, m3 = k->m3;
  if (!(s12 > (m1 + m2) * (m1 + m2) && s12 < (M - m3) * (M - m3))) return 0;
  double m12 = sqrt(s12);
  double E2 = (s12 - m1 * m1 + m2 * m2) / (2 * m12);
  double E3 = (M * M - s12 - m3 * m3) / (2 * m12);
  double p2 = sqrt(fmax(E2 * E2 - m2 * m2, 0.0));
  double p3 = sqrt(fmax(E3 * E3 - m3 * m3, 0.0));
  double s23min = (E2 + E3) * (E2 + E3) - (p2 + p3) * (p2 + p3);
  double s23max = (E2 + E3) * (E2 + E3) - (p2 - p3) * (p2 - p3);
  double s23 = M * M + m1 * m1 + m2 * m2 + m3 * m3 - s12 - s13;
  return s23 >= s23min && s23 <= s23max;
}

/* Invariants of a channel: s_ab, s_bc, s_ac and the masses m_a, m_b, m_c. */
static void channel_invariants(const orc_dkin* k, int ch, double s12, double s13, double* sab,
                               double* sbc, double* sac, double* ma, double* mb, double* mc) {
  double s23 = k->M * k->M + k->m1 * k->m1 + k->m2 * k->m2 + k->m3 * k->m3 - s12 - s13;
  if (ch == 0) { *sab = s12; *sbc = s23; *sac = s13; *ma = k->m1; *mb = k->m2; *mc = k->m3; }
  else if (ch == 1) { *sab = s13; *sbc = s23; *sac = s12; *ma = k->m1; *mb = k->m3; *mc = k->m2; }
  else { *sab = s23; *sbc = s13; *sac = s12; *ma = k->m2; *mb = k->m3; *mc = k->m1; }
}

/* Squared break-up momentum of a, b in their rest frame at invariant mass^2 s. */
static double breakup_q2(double s, double ma, double mb) {
  return (s - (ma + mb) * (ma + mb)) * (s - (ma - mb) * (ma - mb)) / (4 * s);
}

/* Blatt-Weisskopf barrier polynomial B_L(z), z = (qR)^2; F_L(q) = sqrt(B_L(z0)/B_L(z)). */
static double bw_barrier_poly(int L, double z) {
  if (L == 0) return 1.0;
  if (L == 1) return 1.0 + z;
  return 9.0 + 3.0 * z + z * z;
}
static double bw_barrier_poly_dz(int L, double z) {
  if (L == 0) return 0.0;
  if (L == 1) return 1.0;
  return 3.0 + 2.0 * z;
}

/* Zemach spin factor S_L in Lorentz invariants. */
static double zemach(int L, const orc_dkin* k, double sab, double sbc, double sac, double ma,
                     double mb, double mc) {
  if (L == 0) return 1.0;
  double M2 = k->M * k->M;
  double s1 = sbc - sac + (M2 - mc * mc) * (ma * ma - mb * mb) / sab;
  if (L == 1) return s1;
  double a2 = sab - 2 * M2 - 2 * mc * mc + (M2 - mc * mc) * (M2 - mc * mc) / sab;
  double a3 = sab - 2 * ma * ma - 2 * mb * mb + (ma * ma - mb * mb) * (ma * ma - mb * mb) / sab;
  return s1 * s1 - a2 * a3 / 3.0;
}

/* Amplitude of one resonance, A_r = F_L(q) S_L BW(s_ab), with
 *   Gamma(m) = Gamma0 (q/q0)^{2L+1} (m0/m) F_L^2,  BW = 1/(m0^2 - s - i m0 Gamma(m)).
 * If d is not NULL, also dA/dm0 (d[0], d[1]) and dA/dGamma0 (d[2], d[3]). */
void orc_dalitz_amp(const orc_dkin* k, int ch, int L, double m0, double g0, double s12,
                    double s13, double* are, double* aim, double* d) {
  double sab, sbc, sac, ma, mb, mc;
  channel_invariants(k, ch, s12, s13, &sab, &sbc, &sac, &ma, &mb, &mc);
  double m = sqrt(sab);
  double q2 = breakup_q2(sab, ma, mb);
  double q02 = breakup_q2(m0 * m0, ma, mb);
  double q = sqrt(q2), q0 = sqrt(q02);
  double R2 = k->R * k->R;
  double z = q2 * R2, z0 = q02 * R2;
  double F2 = bw_barrier_poly(L, z0) / bw_barrier_poly(L, z);
  double F = sqrt(F2);
  double ratio = pow(q / q0, 2 * L + 1);
  double G = g0 * ratio * (m0 / m) * F2;
  double S = zemach(L, k, sab, sbc, sac, ma, mb, mc);
  /* BW = 1/(dr + i di), dr = m0^2 - s, di = -m0 G */
  double dr = m0 * m0 - sab, di = -m0 * G;
  double dd = dr * dr + di * di;
  double bre = dr / dd, bim = -di / dd;
  *are = F * S * bre;
  *aim = F * S * bim;
  if (d) {
    /* dq0^2/dm0 = (m0^4 - A B)/(2 m0^3), A = (ma+mb)^2, B = (ma-mb)^2 */
    double A = (ma + mb) * (ma + mb), B = (ma - mb) * (ma - mb);
    double dq02 = (m0 * m0 * m0 * m0 - A * B) / (2 * m0 * m0 * m0);
    double dz0 = R2 * dq02;
    double dlogF2 = bw_barrier_poly_dz(L, z0) * dz0 / bw_barrier_poly(L, z0);
    /* dlog Gamma/dm0 = -(2L+1)/2 * dq02/q02 + 1/m0 + dlogF2 */
    double dlogG = -(2 * L + 1) * 0.5 * dq02 / q02 + 1.0 / m0 + dlogF2;
    double dG = G * dlogG;
    /* dD/dm0 = 2 m0 - i (G + m0 dG) */
    double dDr = 2 * m0, dDi = -(G + m0 * dG);
    /* dBW/dm0 = -BW^2 dD/dm0 */
    double b2r = bre * bre - bim * bim, b2i = 2 * bre * bim;
    double dbr = -(b2r * dDr - b2i * dDi), dbi = -(b2r * dDi + b2i * dDr);
    double dF = 0.5 * F * dlogF2;
    d[0] = S * (dF * bre + F * dbr);
    d[1] = S * (dF * bim + F * dbi);
    /* dD/dGamma0 = -i m0 G/g0 -> dBW/dGamma0 = i m0 (G/g0) BW^2 */
    double c = m0 * G / g0;
    d[2] = F * S * (-c * b2i);
    d[3] = F * S * (c * b2r);
  }
}

/* Total amplitude A = a_NR + sum_r c_r A_r at one point; gradient of |A|^2 over all
 * parameters if g != NULL (g has np entries, overwritten). */
static double dalitz_intensity(const orc_dkin* k, int nres, const orc_res* res, const double* p,
                              int np, double anr_re, double anr_im, double s12, double s13,
                              double* g, double* Are_out, double* Aim_out) {
  double Are = anr_re, Aim = anr_im;
  double ar[64], ai[64], dd[64][4];
  for (int r = 0; r < nres; ++r) {
    orc_dalitz_amp(k, res[r].channel, res[r].spin, p[res[r].p_m0], p[res[r].p_g0], s12, s13,
                   &ar[r], &ai[r], g ? dd[r] : NULL);
    double cr = p[res[r].p_re], ci = p[res[r].p_im];
    Are += cr * ar[r] - ci * ai[r];
    Aim += cr * ai[r] + ci * ar[r];
  }
  if (Are_out) { *Are_out = Are; *Aim_out = Aim; }
  if (g) {
    memset(g, 0, sizeof(double) * np);
    for (int r = 0; r < nres; ++r) {
      /* conj(A) A_r */
      double xr = Are * ar[r] + Aim * ai[r];
      double xi = Are * ai[r] - Aim * ar[r];
      g[res[r].p_re] += 2 * xr;
      g[res[r].p_im] += -2 * xi;
      double cr = p[res[r].p_re], ci = p[res[r].p_im];
      /* 2 Re(conj(A) c_r dA_r) */
      double um = cr * dd[r][0] - ci * dd[r][1], vm = cr * dd[r][1] + ci * dd[r][0];
      g[res[r].p_m0] += 2 * (Are * um + Aim * vm);
      double ug = cr * dd[r][2] - ci * dd[r][3], vg = cr * dd[r][3] + ci * dd[r][2];
      g[res[r].p_g0] += 2 * (Are * ug + Aim * vg);
    }
  }
  return Are * Are + Aim * Aim;
}

/* Grid bounds: s12 in [(m1+m2)^2, (M-m3)^2], s13 in [(m1+m3)^2, (M-m2)^2]. */
static void dalitz_box(const orc_dkin* k, double* x0, double* x1, double* y0, double* y1) {
  *x0 = (k->m1 + k->m2) * (k->m1 + k->m2);
  *x1 = (k->M - k->m3) * (k->M - k->m3);
  *y0 = (k->m1 + k->m3) * (k->m1 + k->m3);
  *y1 = (k->M - k->m2) * (k->M - k->m2);
}

/* Normalisation N = dA * sum over cells whose centre is inside |A(centre)|^2, and dN
 * over all parameters; ncells gets the number of cells inside. */
int orc_dalitz_norm(const orc_dkin* k, int nres, const orc_res* res, const double* p, int np,
                    double anr_re, double anr_im, int nbx, int nby, double* N, double* dN,
                    int64_t* ncells) {
  double x0, x1, y0, y1;
  dalitz_box(k, &x0, &x1, &y0, &y1);
  double hx = (x1 - x0) / nbx, hy = (y1 - y0) / nby;
  orc_acc s = {0, 0};
  orc_acc* gs = (orc_acc*)calloc(np, sizeof(orc_acc));
  double* g = (double*)malloc(sizeof(double) * np);
  int64_t cnt = 0;
  for (int i = 0; i < nbx; ++i) {
    double s12 = x0 + (i + 0.5) * hx;
    for (int j = 0; j < nby; ++j) {
      double s13 = y0 + (j + 0.5) * hy;
      if (!orc_dalitz_inside(k, s12, s13)) continue;
      ++cnt;
      double P = dalitz_intensity(k, nres, res, p, np, anr_re, anr_im, s12, s13, dN ? g : NULL,
                                  NULL, NULL);
      acc_add(&s, P);
      if (dN) for (int q = 0; q < np; ++q) acc_add(&gs[q], g[q]);
    }
  }
  *N = hx * hy * acc_get(&s);
  if (dN) for (int q = 0; q < np; ++q) dN[q] = hx * hy * acc_get(&gs[q]);
  if (ncells) *ncells = cnt;
  free(gs);
  free(g);
  return 0;
}

/* Per-event |A|^2 and the interference condition number
 * kappa = (|a_NR| + sum |c_r A_r|)^2 / |A|^2. */
int orc_dalitz_intensity(const orc_dkin* k, int nres, const orc_res* res, const double* p, int np,
                         double anr_re, double anr_im, int64_t n, const double* s12,
                         const double* s13, double* P, double* kappa) {
  (void)np;
  for (int64_t i = 0; i < n; ++i) {
    double Are, Aim;
    P[i] = dalitz_intensity(k, nres, res, p, np, anr_re, anr_im, s12[i], s13[i], NULL, &Are, &Aim);
    if (kappa) {
      double sum = hypot(anr_re, anr_im);
      for (int r = 0; r < nres; ++r) {
        double ar, ai;
        orc_dalitz_amp(k, res[r].channel, res[r].spin, p[res[r].p_m0], p[res[r].p_g0], s12[i],
                       s13[i], &ar, &ai, NULL);
        sum += hypot(ar, ai) * hypot(p[res[r].p_re], p[res[r].p_im]);
      }
      kappa[i] = sum * sum / P[i];
    }
  }
  return 0;
}

/* NLL = -sum_i log |A_i|^2 + n log N, with the gradient over all np parameters. */
int orc_dalitz_nll(const orc_dkin* k, int nres, const orc_res* res, const double* p, int np,
                   double anr_re, double anr_im, int nbx, int nby, int64_t n, const double* s12,
                   const double* s13, double* nll, double* grad) {
  double N;
  double* dN = grad ? (double*)malloc(sizeof(double) * np) : NULL;
  orc_dalitz_norm(k, nres, res, p, np, anr_re, anr_im, nbx, nby, &N, dN, NULL);
  orc_acc s = {0, 0};
  orc_acc* gs = (orc_acc*)calloc(np, sizeof(orc_acc));
  double* g = (double*)malloc(sizeof(double) * np);
  for (int64_t i = 0; i < n; ++i) {
    double P = dalitz_intensity(k, nres, res, p, np, anr_re, anr_im, s12[i], s13[i],
                                grad ? g : NULL, NULL, NULL);
    acc_add(&s, -log(P));
    if (grad) for (int q = 0; q < np; ++q) acc_add(&gs[q], -g[q] / P);
  }
  *nll = acc_get(&s) + (double)n * log(N);
  if (grad) for (int q = 0; q < np; ++q) grad[q] = acc_get(&gs[q]) + (double)n * dN[q] / N;
  free(gs);
  free(g);
  free(dN);
  return 0;
}

/* ------------------------------------------------------------------------------ */
/* Array helpers for the Python wrapper (loops over the scalar definitions above).  */
/* ------------------------------------------------------------------------------ */
void orc_faddeeva_many(int64_t n, const double* x, const double* y, double* re, double* im) {
  for (int64_t i = 0; i < n; ++i) orc_faddeeva(x[i], y[i], &re[i], &im[i]);
}

void orc_leaf_shape_many(const orc_node* nd, const double* p, int64_t n, const double* x,
                         double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = leaf_shape(nd, p, x[i], NULL);
}

void orc_dalitz_inside_many(const orc_dkin* k, int64_t n, const double* s12, const double* s13,
                            int8_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = (int8_t)orc_dalitz_inside(k, s12[i], s13[i]);
}

void orc_dalitz_amp_many(const orc_dkin* k, int ch, int L, double m0, double g0, int64_t n,
                         const double* s12, const double* s13, double* re, double* im,
                         double* d /* n x 4 or NULL */) {
  for (int64_t i = 0; i < n; ++i)
    orc_dalitz_amp(k, ch, L, m0, g0, s12[i], s13[i], &re[i], &im[i], d ? d + 4 * i : NULL);
}

/* Zemach factor of one channel at a point, for pins against explicit four-vectors. */
double orc_zemach_at(const orc_dkin* k, int ch, int L, double s12, double s13) {
  double sab, sbc, sac, ma, mb, mc;
  channel_invariants(k, ch, s12, s13, &sab, &sbc, &sac, &ma, &mb, &mc);
  return zemach(L, k, sab, sbc, sac, ma, mb, mc);
}

/* ------------------------------------------------------------------------------ */
/* Time-dependent Dalitz model (Sec. 4: the D0 -> pi+ pi- pi0 mixing fit, whose time */
/* dependence is cosh/sinh and cos/sin terms, each smeared by a Gaussian resolution, */
/* with a per-event decay-time uncertainty).  The paper gives no formula;           */
/* the reading used here is the standard one for D0 mixing in a self-conjugate       */
/* multi-body final state, with q/p = 1:                                           */
/*   I(s12, s13, t) = 1/2 (|A|^2 + |B|^2) Tch + 1/2 (|A|^2 - |B|^2) Tc               */
/*                    + Re(A* B) Tsh - Im(A* B) Ts,                                  */
/* A = a_NR + sum_r c_r A_r(s12, s13) the D0 amplitude, B the D0bar amplitude, the   */
/* same sum at the CP-conjugate point (1 <-> 2 exchanged: s13 <-> s23), and the time  */
/* factors e^{-Gt} {cosh yGt, cos xGt, sinh yGt, sin xGt} each convolved with a      */
/* Gaussian of width sigma = s sigma_t (sigma_t per event, s a scale parameter):     */
/*   Tch = (T(l1) + T(l2))/2, Tsh = (T(l1) - T(l2))/2, Tc + i Ts = T(l3),            */
/*   l1 = G(1 - y), l2 = G(1 + y), l3 = G(1 - i x), G = 1/tau,                       */
/*   T(l) = Int_0^inf e^{-l u} Gauss(t - u; sigma) du.                               */
/* Normalised over the Dalitz region (cell centres of the nbx x nby grid) and all t: */
/*   N = dA sum_cells [1/2 (|A|^2 + |B|^2) Ich + 1/2 (|A|^2 - |B|^2) Ic             */
/*                     + Re(A* B) Ish - Im(A* B) Is],                                */
/* Ich = (1/l1 + 1/l2)/2, Ish = (1/l1 - 1/l2)/2, Ic + i Is = 1/l3 (the time          */
/* integrals over the real line; independent of sigma).  P = I/N; conditional on    */
/* sigma_t (no sigma_t density).                                                     */
/* ------------------------------------------------------------------------------ */
#include <complex.h>

typedef struct {
  int32_t p_tau, p_x, p_y, p_s;
  int32_t dens;            /* 1: the sigma_t density below is part of the PDF          */
  int32_t p_b0, p_b1, p_b2; /* its parameters                                           */
  double slo, shi;         /* the sigma_t range                                        */
} orc_tpar;

/* ------------------------------------------------------------------------------ */
/* The decay-time uncertainty's density (Sec. 4: the sigma_t distribution of the    */
/* mixing fit varies across the Dalitz plot; the paper gives no form).  Reading: a  */
/* Gamma distribution of shape 2 truncated to [slo, shi], whose rate varies         */
/* log-linearly over the plot:                                                       */
/*   D(st | s12, s13) = lam^2 st e^{-lam st} / Z(lam),                               */
/*   lam = exp(b0 + b1 (s12 - sc) + b2 (s13 - sc)),  sc = (M^2 + m1^2 + m2^2 + m3^2)/3, */
/*   Z = g(lam slo) - g(lam shi),  g(a) = e^{-a} (1 + a)  (the integral of the shape). */
/* The full PDF is I/N times D: D integrates to one over st at every point, so the  */
/* product is normalised over (s12, s13, t, st).                                     */
/* ------------------------------------------------------------------------------ */
static double sigt_logd(const orc_dkin* k, const orc_tpar* tp, const double* p, double s12,
                        double s13, double st, double* g3) {
  double sc = (k->M * k->M + k->m1 * k->m1 + k->m2 * k->m2 + k->m3 * k->m3) / 3.0;
  double u = s12 - sc, v = s13 - sc;
  double ll = p[tp->p_b0] + p[tp->p_b1] * u + p[tp->p_b2] * v;
  double lam = exp(ll);
  double el = exp(-lam * tp->slo), eh = exp(-lam * tp->shi);
  double Z = el * (1.0 + lam * tp->slo) - eh * (1.0 + lam * tp->shi);
  if (g3) {
    /* dZ/dlam = -lam slo^2 e^{-lam slo} + lam shi^2 e^{-lam shi} */
    double dZ = -lam * tp->slo * tp->slo * el + lam * tp->shi * tp->shi * eh;
    double dl = 2.0 / lam - st - dZ / Z; /* d log D / d lam */
    g3[0] = dl * lam;
    g3[1] = dl * lam * u;
    g3[2] = dl * lam * v;
  }
  return 2.0 * ll + log(st) - lam * st - log(Z);
}

void orc_sigt_logd_many(const orc_dkin* k, const orc_tpar* tp, const double* p, int64_t n,
                        const double* s12, const double* s13, const double* st, double* out,
                        double* g /* n x 3 or NULL */) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = sigt_logd(k, tp, p, s12[i], s13[i], st[i], g ? g + 3 * i : NULL);
}

/* w(z) for any z: the Im z > 0 routine, w(z) = 2 e^{-z^2} - w(-z) below the axis. */
static double complex faddeeva_any(double complex z) {
  double re, im;
  if (cimag(z) > 0) {
    orc_faddeeva(creal(z), cimag(z), &re, &im);
    return re + I * im;
  }
  orc_faddeeva(-creal(z), -cimag(z), &re, &im);
  return 2.0 * cexp(-z * z) - (re + I * im);
}

/* T(l; t, sigma) = 1/2 e^{l^2 sigma^2/2 - l t} erfc((l sigma^2 - t)/(sigma sqrt2))
 *               = 1/2 e^{-t^2/(2 sigma^2)} w(i u),  u = (l sigma^2 - t)/(sigma sqrt2),
 * using w(i u) = e^{u^2} erfc(u); for Re u < 0 the reflection gives
 * T = e^{l^2 sigma^2/2 - l t} - 1/2 e^{-t^2/(2 sigma^2)} w(-i u).
 * dT/dl = (l sigma^2 - t) T - sigma/sqrt(2 pi) e^{-t^2/(2 sigma^2)},
 * dT/dsigma = l^2 sigma T - e^{-t^2/(2 sigma^2)} (l sigma^2 + t)/(sqrt(2 pi) sigma^2). */
static double complex smeared_exp(double complex l, double t, double sig, double complex* dl,
                                  double complex* ds) {
  double complex u = (l * sig * sig - t) / (sig * ORC_SQRT2);
  double g = exp(-t * t / (2 * sig * sig));
  double complex T;
  if (creal(u) >= 0) T = 0.5 * g * faddeeva_any(I * u);
  else T = cexp(l * l * sig * sig / 2 - l * t) - 0.5 * g * faddeeva_any(-I * u);
  if (dl) *dl = (l * sig * sig - t) * T - sig / sqrt(2 * ORC_PI) * g;
  if (ds) *ds = l * l * sig * T - g * (l * sig * sig + t) / (sqrt(2 * ORC_PI) * sig * sig);
  return T;
}

void orc_smeared_exp_many(int64_t n, double lr, double li, const double* t, double sig,
                          double* Tr, double* Ti) {
  for (int64_t i = 0; i < n; ++i) {
    double complex T = smeared_exp(lr + I * li, t[i], sig, NULL, NULL);
    Tr[i] = creal(T);
    Ti[i] = cimag(T);
  }
}

/* Amplitudes A (at (s12, s13)) and B (at (s12, s23)) with their coefficient derivatives:
 * a[r], b[r] the per-resonance amplitudes (A = 1 + sum c_r a_r). */
static void tddp_amps(const orc_dkin* k, int nres, const orc_res* res, const double* p,
                      double s12, double s13, double complex* A, double complex* B,
                      double complex* a, double complex* b, double complex (*da)[2],
                      double complex (*db)[2]) {
  double s23 = k->M * k->M + k->m1 * k->m1 + k->m2 * k->m2 + k->m3 * k->m3 - s12 - s13;
  *A = 1.0;
  *B = 1.0;
  for (int r = 0; r < nres; ++r) {
    double re, im, d[4];
    orc_dalitz_amp(k, res[r].channel, res[r].spin, p[res[r].p_m0], p[res[r].p_g0], s12, s13,
                   &re, &im, da ? d : NULL);
    a[r] = re + I * im;
    if (da) {
      da[r][0] = d[0] + I * d[1];
      da[r][1] = d[2] + I * d[3];
    }
    orc_dalitz_amp(k, res[r].channel, res[r].spin, p[res[r].p_m0], p[res[r].p_g0], s12, s23,
                   &re, &im, db ? d : NULL);
    b[r] = re + I * im;
    if (db) {
      db[r][0] = d[0] + I * d[1];
      db[r][1] = d[2] + I * d[3];
    }
    double complex c = p[res[r].p_re] + I * p[res[r].p_im];
    *A += c * a[r];
    *B += c * b[r];
  }
}

/* Change of h(A, B) below for a change (dA, dB) of the amplitudes. */
static double tddp_dh(double complex A, double complex B, double complex dA, double complex dB,
                      const double* kk) {
  double daa = 2 * creal(conj(A) * dA), dbb = 2 * creal(conj(B) * dB);
  double complex dx = conj(dA) * B + conj(A) * dB;
  return 0.5 * (daa + dbb) * kk[0] + 0.5 * (daa - dbb) * kk[1] + creal(dx) * kk[2] -
         cimag(dx) * kk[3];
}

/* The four time coefficients and the combination h(A, B) = 1/2 (|A|^2 + |B|^2) k0 +
 * 1/2 (|A|^2 - |B|^2) k1 + Re(A* B) k2 - Im(A* B) k3, with its derivatives in the
 * coefficients c_r and (da, db not NULL) in the resonance masses and widths (added to g
 * scaled by w) and in the k's (returned in dk[4]). */
static double tddp_comb(int nres, const orc_res* res, const double* p, double complex A,
                        double complex B, const double complex* a, const double complex* b,
                        double complex (*da)[2], double complex (*db)[2], const double* kk,
                        double w, double* g, double* dk) {
  double aa = creal(A) * creal(A) + cimag(A) * cimag(A);
  double bb = creal(B) * creal(B) + cimag(B) * cimag(B);
  double complex x = conj(A) * B;
  if (dk) {
    dk[0] = 0.5 * (aa + bb);
    dk[1] = 0.5 * (aa - bb);
    dk[2] = creal(x);
    dk[3] = -cimag(x);
  }
  if (g)
    for (int r = 0; r < nres; ++r) {
      for (int part = 0; part < 2; ++part) {
        double complex dA = part ? I * a[r] : a[r], dB = part ? I * b[r] : b[r];
        g[part ? res[r].p_im : res[r].p_re] += w * tddp_dh(A, B, dA, dB, kk);
      }
      if (da && db) {
        /* dA = c_r da_r/dm0 (dGamma0), dB likewise */
        double complex c = p[res[r].p_re] + I * p[res[r].p_im];
        g[res[r].p_m0] += w * tddp_dh(A, B, c * da[r][0], c * db[r][0], kk);
        g[res[r].p_g0] += w * tddp_dh(A, B, c * da[r][1], c * db[r][1], kk);
      }
    }
  return 0.5 * (aa + bb) * kk[0] + 0.5 * (aa - bb) * kk[1] + creal(x) * kk[2] - cimag(x) * kk[3];
}

/* Time coefficients of an event (T's) or of the normalisation (integrals), and their
 * derivatives d k_j / d(tau, x, y, s) in dkk[j][0..3]. */
static void tddp_time(const double* p, const orc_tpar* tp, double t, double sigt, int integral,
                      double* kk, double dkk[4][4]) {
  double tau = p[tp->p_tau], x = p[tp->p_x], y = p[tp->p_y], s = p[tp->p_s];
  double G = 1.0 / tau;
  double complex l[3] = {G * (1 - y), G * (1 + y), G * (1 - I * x)};
  /* dl/dtau, dl/dx, dl/dy */
  double complex dlt[3] = {-(1 - y) * G * G, -(1 + y) * G * G, -(1 - I * x) * G * G};
  double complex dlx[3] = {0, 0, -I * G};
  double complex dly[3] = {-G, G, 0};
  double complex T[3], Tl[3], Ts[3];
  double sig = s * sigt;
  for (int j = 0; j < 3; ++j) {
    if (integral) {
      T[j] = 1.0 / l[j];
      Tl[j] = -1.0 / (l[j] * l[j]);
      Ts[j] = 0;
    } else {
      T[j] = smeared_exp(l[j], t, sig, &Tl[j], &Ts[j]);
      Ts[j] *= sigt; /* d/ds */
    }
  }
  kk[0] = 0.5 * creal(T[0] + T[1]);
  kk[2] = 0.5 * creal(T[0] - T[1]);
  kk[1] = creal(T[2]);
  kk[3] = cimag(T[2]);
  for (int q = 0; q < 4; ++q) {
    double complex d[3];
    for (int j = 0; j < 3; ++j)
      d[j] = q == 0 ? Tl[j] * dlt[j] : q == 1 ? Tl[j] * dlx[j] : q == 2 ? Tl[j] * dly[j] : Ts[j];
    dkk[0][q] = 0.5 * creal(d[0] + d[1]);
    dkk[2][q] = 0.5 * creal(d[0] - d[1]);
    dkk[1][q] = creal(d[2]);
    dkk[3][q] = cimag(d[2]);
  }
}

/* Normalisation N and its gradient (cell centres inside the region, dA per cell). */
static double tddp_norm(const orc_dkin* k, int nres, const orc_res* res, const orc_tpar* tp,
                        const double* p, int np, int nbx, int nby, double* dN) {
  double x0, x1, y0, y1;
  dalitz_box(k, &x0, &x1, &y0, &y1);
  double hx = (x1 - x0) / nbx, hy = (y1 - y0) / nby, dA = hx * hy;
  double kk[4], dkk[4][4];
  tddp_time(p, tp, 0, 1, 1, kk, dkk);
  orc_acc s = {0, 0};
  orc_acc* gs = (orc_acc*)calloc(np, sizeof(orc_acc));
  orc_acc sk[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  double* g = (double*)malloc(sizeof(double) * np);
  double complex a[64], b[64], da[64][2], db[64][2], A, B;
  for (int i = 0; i < nbx; ++i)
    for (int j = 0; j < nby; ++j) {
      double s12 = x0 + (i + 0.5) * hx, s13 = y0 + (j + 0.5) * hy;
      if (!orc_dalitz_inside(k, s12, s13)) continue;
      tddp_amps(k, nres, res, p, s12, s13, &A, &B, a, b, dN ? da : NULL, dN ? db : NULL);
      double dk[4];
      memset(g, 0, sizeof(double) * np);
      acc_add(&s, tddp_comb(nres, res, p, A, B, a, b, dN ? da : NULL, dN ? db : NULL, kk, 1.0,
                            dN ? g : NULL, dk));
      if (dN) {
        for (int q = 0; q < np; ++q) acc_add(&gs[q], g[q]);
        for (int j = 0; j < 4; ++j) acc_add(&sk[j], dk[j]);
      }
    }
  if (dN) {
    for (int q = 0; q < np; ++q) dN[q] = dA * acc_get(&gs[q]);
    int ip[4] = {tp->p_tau, tp->p_x, tp->p_y, tp->p_s};
    for (int q = 0; q < 4; ++q)
      for (int j = 0; j < 4; ++j) dN[ip[q]] += dA * acc_get(&sk[j]) * dkk[j][q];
  }
  free(gs);
  free(g);
  return dA * acc_get(&s);
}

/* Per-event intensity I (unnormalised) with gradient g (optional). */
static double tddp_event(const orc_dkin* k, int nres, const orc_res* res, const orc_tpar* tp,
                         const double* p, int np, double s12, double s13, double t, double sigt,
                         double* g) {
  double kk[4], dkk[4][4], dk[4];
  tddp_time(p, tp, t, sigt, 0, kk, dkk);
  double complex a[64], b[64], da[64][2], db[64][2], A, B;
  tddp_amps(k, nres, res, p, s12, s13, &A, &B, a, b, g ? da : NULL, g ? db : NULL);
  if (g) memset(g, 0, sizeof(double) * np);
  double v = tddp_comb(nres, res, p, A, B, a, b, g ? da : NULL, g ? db : NULL, kk, 1.0, g, dk);
  if (g) {
    int ip[4] = {tp->p_tau, tp->p_x, tp->p_y, tp->p_s};
    for (int q = 0; q < 4; ++q)
      for (int j = 0; j < 4; ++j) g[ip[q]] += dk[j] * dkk[j][q];
  }
  return v;
}

int orc_tddp_intensity(const orc_dkin* k, int nres, const orc_res* res, const orc_tpar* tp,
                       const double* p, int np, int64_t n, const double* s12, const double* s13,
                       const double* t, const double* sigt, double* out) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = tddp_event(k, nres, res, tp, p, np, s12[i], s13[i], t[i], sigt[i], NULL);
  return 0;
}

double orc_tddp_norm(const orc_dkin* k, int nres, const orc_res* res, const orc_tpar* tp,
                     const double* p, int np, int nbx, int nby, double* dN) {
  return tddp_norm(k, nres, res, tp, p, np, nbx, nby, dN);
}

/* NLL = -sum_i log(I_i / N) and its gradient. */
int orc_tddp_nll(const orc_dkin* k, int nres, const orc_res* res, const orc_tpar* tp,
                 const double* p, int np, int nbx, int nby, int64_t n, const double* s12,
                 const double* s13, const double* t, const double* sigt, double* nll,
                 double* grad) {
  double* dN = grad ? (double*)calloc(np, sizeof(double)) : NULL;
  double N = tddp_norm(k, nres, res, tp, p, np, nbx, nby, dN);
  orc_acc s = {0, 0};
  orc_acc* gs = (orc_acc*)calloc(np, sizeof(orc_acc));
  double* g = (double*)malloc(sizeof(double) * np);
  for (int64_t i = 0; i < n; ++i) {
    double v = tddp_event(k, nres, res, tp, p, np, s12[i], s13[i], t[i], sigt[i], grad ? g : NULL);
    acc_add(&s, -log(v));
    if (grad) for (int q = 0; q < np; ++q) acc_add(&gs[q], -g[q] / v);
    if (tp->dens) {
      double g3[3];
      acc_add(&s, -sigt_logd(k, tp, p, s12[i], s13[i], sigt[i], grad ? g3 : NULL));
      if (grad) {
        acc_add(&gs[tp->p_b0], -g3[0]);
        acc_add(&gs[tp->p_b1], -g3[1]);
        acc_add(&gs[tp->p_b2], -g3[2]);
      }
    }
  }
  *nll = acc_get(&s) + (double)n * log(N);
  if (grad) for (int q = 0; q < np; ++q) grad[q] = acc_get(&gs[q]) + (double)n * dN[q] / N;
  free(gs);
  free(g);
  free(dN);
  return 0;
}
