// FP64 CPU oracle for the ARCHER-NM internal-dosimetry Monte Carlo
// (Peng et al., "Development of a GPU-accelerated Monte Carlo dose calculation
// module for nuclear medicine, ARCHER-NM", §2.1, Eq. 1-3).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference
// that the CUDA path is checked against.  Only the test suite, the package's
// smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
// code, header, table or constant generator with the CUDA path; the physics
// constants below are restated here from their published definitions.
//
// The method is a stochastic transport iteration, not a closed form, so the
// oracle follows the paper's steps with independent sub-algorithms that have the
// same distributions as the GPU's:
//   * decay voxel: inverse CDF over the PET-derived activity (§2.1, linear
//     PET -> decay PDF), binary search in an FP64 cumulative table;
//   * directions: Marsaglia's 1972 sphere method (§2.1);
//   * free flight: exact voxel traversal (Siddon's parametric plane-crossing
//     form, walked incrementally) against a sampled optical depth -- no Woodcock;
//   * Compton: rejection sampling straight from the Klein-Nishina dσ/dΩ -- no
//     Kahn; photoelectric absorption; optional Rayleigh (Thomson shape); photon
//     cutoff with local deposition of the remainder (§2.1);
//   * RNG: std::mt19937_64, seeded per chunk of histories;
//   * tallies: int64 fixed point, one unit = 2^-6 eV, every deposit a difference
//     q(E_before) - q(E_after) so that energy conservation is exact;
//   * positron (optional): kinetic energy by rejection from the allowed beta+
//     spectrum with the Fermi function, a straight track that uses up the Katz-
//     Penfold mass range voxel by voxel, annihilation at its end;
//   * statistics: batch means over B batches, Eq. 1 dose rate, Eq. 2 organ means,
//     Eq. 3 organ RMS relative uncertainty, batch sigma of the organ means; and,
//     on request, the history-by-history sigma (§2.1's method, Walters et al.
//     2002): each history's total deposit per voxel is squared and summed.
//
// Functions that no closed form or invariant pins are marked "parity unpinned"
// at their definition (none at present): the decay-voxel inverse CDF inside
// orc_run is pinned by a chi-square test of its decay counts, the interaction
// choice and the Compton kinematics through interact() (which orc_run calls)
// by binomial and closed-form tests, and the Thomson sampler by chi-square.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <thread>
#include <vector>

namespace {

// Physical constants (CODATA 2018 values).
constexpr double kElectronMassMeV = 0.51099895;       // m_e c^2
constexpr double kClassicalRadiusCm = 2.8179403262e-13;  // r_e
constexpr double kAvogadro = 6.02214076e23;
constexpr double kJoulePerEv = 1.602176634e-19;
constexpr double kPi = 3.14159265358979323846;
constexpr double kFineStructure = 7.2973525693e-3;     // alpha
// Tally unit: 2^-6 eV, so 1 MeV = 6.4e7 units.
constexpr double kUnitsPerMeV = 64.0e6;

inline int64_t q_units(double e_mev) { return (int64_t)std::llrint(e_mev * kUnitsPerMeV); }

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Cross sections (§2.1: photoelectric and Compton explicit, pair production
// absent below 1.02 MeV).
// ---------------------------------------------------------------------------

// Klein-Nishina total cross section per electron, cm^2 (closed form).
double orc_sigma_kn(double e_mev) {
  const double k = e_mev / kElectronMassMeV;
  const double a = 1.0 + 2.0 * k;
  const double l = std::log1p(2.0 * k);  // ln(1 + 2k) without rounding 1 + 2k first
  const double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k);
  const double t2 = l / (2.0 * k);
  const double t3 = (1.0 + 3.0 * k) / (a * a);
  return 2.0 * kPi * kClassicalRadiusCm * kClassicalRadiusCm * (t1 + t2 - t3);
}

// Klein-Nishina differential cross section per electron, cm^2/sr, at scattering
// cosine c: (r_e^2/2) P^2 (P + 1/P - sin^2θ), with P = E'/E.
double orc_dsigma_kn(double e_mev, double c) {
  const double k = e_mev / kElectronMassMeV;
  const double p = 1.0 / (1.0 + k * (1.0 - c));
  return 0.5 * kClassicalRadiusCm * kClassicalRadiusCm * p * p * (p + 1.0 / p - (1.0 - c * c));
}

typedef struct {
  int32_t n;                 // number of materials
  const double* z_over_a;    // [n] electrons per unit mass: rho * N_A * Z/A electrons per cm^3
  const double* zeff;        // [n] effective atomic number for the photoelectric term
  double pe_coeff;           // C in mu_pe/rho = C * Zeff^pe_exp / E^3   (cm^2/g MeV^3)
  double pe_exp;             // 3.8
  double rayleigh_coeff;     // c_R in mu_R/rho = c_R * Zeff^2 / E^2    (cm^2/g MeV^2)
  int32_t rayleigh;          // 0 = off (paper), 1 = on
  double photon_cut_mev;     // 0.010 (§2.1)
} orc_materials;

// Mass attenuation coefficients (cm^2/g) of material m at energy E: Compton
// (electrons per gram N_A Z/A times sigma_KN), photoelectric, Rayleigh.
void orc_mass_atten(const orc_materials* mt, int m, double e_mev, double* c, double* pe,
                    double* r) {
  *c = kAvogadro * mt->z_over_a[m] * orc_sigma_kn(e_mev);
  *pe = mt->pe_coeff * std::pow(mt->zeff[m], mt->pe_exp) / (e_mev * e_mev * e_mev);
  *r = mt->rayleigh ? mt->rayleigh_coeff * mt->zeff[m] * mt->zeff[m] / (e_mev * e_mev) : 0.0;
}

// Linear attenuation coefficients (1/cm) of material m at density rho and energy E.
void orc_mu(const orc_materials* mt, int m, double rho, double e_mev, double* mu_c,
            double* mu_pe, double* mu_r) {
  orc_mass_atten(mt, m, e_mev, mu_c, mu_pe, mu_r);
  *mu_c *= rho;
  *mu_pe *= rho;
  *mu_r *= rho;
}

// ---------------------------------------------------------------------------
// CT -> phantom (§2.1): HU -> mass density by a piecewise-linear curve through
// five (HU, rho) nodes, clamped at the ends; the material is the node nearest
// in HU (ties go to the lower node).  Materials: 0 air, 1 lung, 2 adipose,
// 3 soft tissue, 4 bone.
// ---------------------------------------------------------------------------
void orc_hu_to_phantom(const int16_t* hu, int64_t n, double* density, uint8_t* material) {
  static const double node_hu[5] = {-1000.0, -750.0, -100.0, 40.0, 1000.0};
  static const double node_rho[5] = {0.0012, 0.26, 0.95, 1.03, 1.85};
  for (int64_t i = 0; i < n; ++i) {
    const double h = (double)hu[i];
    double rho;
    if (h <= node_hu[0]) {
      rho = node_rho[0];
    } else if (h >= node_hu[4]) {
      rho = node_rho[4];
    } else {
      int s = 0;
      while (!(h >= node_hu[s] && h <= node_hu[s + 1])) ++s;
      const double f = (h - node_hu[s]) / (node_hu[s + 1] - node_hu[s]);
      rho = node_rho[s] + f * (node_rho[s + 1] - node_rho[s]);
    }
    int best = 0;
    double bestd = std::fabs(h - node_hu[0]);
    for (int s = 1; s < 5; ++s) {
      const double d = std::fabs(h - node_hu[s]);
      if (d < bestd) { bestd = d; best = s; }
    }
    density[i] = rho;
    material[i] = (uint8_t)best;
  }
}

// ---------------------------------------------------------------------------
// Sampling primitives.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct Rng {
  std::mt19937_64 g;
  // Uniform in the open interval (0, 1).
  double u() { return ((double)(g() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
};

// Marsaglia (1972): pick (v1, v2) uniform in the unit disc, then map to the sphere.
void marsaglia(Rng& r, double d[3]) {
  double v1, v2, s;
  do {
    v1 = 2.0 * r.u() - 1.0;
    v2 = 2.0 * r.u() - 1.0;
    s = v1 * v1 + v2 * v2;
  } while (s >= 1.0);
  const double f = 2.0 * std::sqrt(1.0 - s);
  d[0] = v1 * f;
  d[1] = v2 * f;
  d[2] = 1.0 - 2.0 * s;
}

// Scattering cosine by rejection from dσ/dΩ: cosθ uniform on [-1, 1] (uniform in
// solid angle), accepted with probability f(c)/2, f = P^2 (P + 1/P - sin^2θ) <= 2.
double sample_kn_cos(Rng& r, double e_mev) {
  const double k = e_mev / kElectronMassMeV;
  for (;;) {
    const double c = 2.0 * r.u() - 1.0;
    const double p = 1.0 / (1.0 + k * (1.0 - c));
    const double f = p * p * (p + 1.0 / p - (1.0 - c * c));
    if (2.0 * r.u() <= f) return c;
  }
}

// Rayleigh scattering cosine with the Thomson shape (1 + c^2)/2 by rejection.
double sample_thomson_cos(Rng& r) {
  for (;;) {
    const double c = 2.0 * r.u() - 1.0;
    if (2.0 * r.u() <= 1.0 + c * c) return c;
  }
}

// New direction at polar cosine c and azimuth phi about d, built from an
// orthonormal frame (e1, e2, d).
void rotate(double d[3], double c, double phi) {
  // Helper axis: the coordinate axis least aligned with d.
  int a = 0;
  if (std::fabs(d[1]) < std::fabs(d[a])) a = 1;
  if (std::fabs(d[2]) < std::fabs(d[a])) a = 2;
  double h[3] = {0.0, 0.0, 0.0};
  h[a] = 1.0;
  double e1[3] = {h[1] * d[2] - h[2] * d[1], h[2] * d[0] - h[0] * d[2], h[0] * d[1] - h[1] * d[0]};
  const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (double& x : e1) x /= n1;
  const double e2[3] = {d[1] * e1[2] - d[2] * e1[1], d[2] * e1[0] - d[0] * e1[2],
                        d[0] * e1[1] - d[1] * e1[0]};
  const double s = std::sqrt(std::max(0.0, 1.0 - c * c));
  const double cp = std::cos(phi), sp = std::sin(phi);
  double nd[3];
  for (int i = 0; i < 3; ++i) nd[i] = c * d[i] + s * (cp * e1[i] + sp * e2[i]);
  const double nn = std::sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
  for (int i = 0; i < 3; ++i) d[i] = nd[i] / nn;
}

// One real interaction of a photon of energy e (MeV) in material m at
// density rho (§2.1: photoelectric and Compton explicit; Rayleigh optional).
// The type is drawn in proportion to the linear attenuation coefficients
// mu_c : mu_pe : mu_R; Compton takes a Klein-Nishina cosine and leaves the
// photon E' = E / (1 + k (1 - cos)), k = E / m_e c^2 (the recoil electron
// keeps E - E'); photoelectric absorption leaves nothing; Rayleigh takes a
// Thomson cosine and keeps E.  Writes the photon's energy after the event
// (0 when absorbed), the scattering cosine and the azimuth.
enum { kCompton = 0, kPhoto = 1, kRayleigh = 2 };

int interact(Rng& r, const orc_materials* mt, int m, double rho, double e, double* e2, double* cth,
             double* phi) {
  double mc, mp, mr;
  orc_mu(mt, m, rho, e, &mc, &mp, &mr);
  const double x = r.u() * (mc + mp + mr);
  *cth = 1.0;
  *phi = 0.0;
  if (x < mc) {
    *cth = sample_kn_cos(r, e);
    const double k = e / kElectronMassMeV;
    *e2 = e / (1.0 + k * (1.0 - *cth));
    *phi = 2.0 * kPi * r.u();
    return kCompton;
  }
  if (x < mc + mp) {
    *e2 = 0.0;
    return kPhoto;
  }
  *cth = sample_thomson_cos(r);
  *phi = 2.0 * kPi * r.u();
  *e2 = e;
  return kRayleigh;
}

struct Grid {
  int nx, ny, nz;
  double d[3];
  const double* density;
  const uint8_t* material;
};

// Voxel index of a point along one axis: floor(p / d), a point on a plane going
// to the upper voxel; -1 or n means outside.
inline int axis_index(double p, double d, int n) {
  if (!(p >= 0.0)) return -1;
  const double f = std::floor(p / d);
  if (f >= (double)n) return n;
  return (int)f;
}

// Exact traversal of the ray p + t*dir (t >= 0) through the voxel grid, in
// Siddon's parametric form: per axis the parameter of the next plane crossing
// and the parameter step between planes; each voxel visit covers [t, t_exit).
// For every visited voxel the callback gets (voxel, t_enter, t_exit) and may
// stop the walk by returning false.  Returns true if the ray left the grid.
template <class F>
bool traverse(const Grid& g, const double p[3], const double dir[3], F&& visit) {
  const int n[3] = {g.nx, g.ny, g.nz};
  int idx[3];
  for (int a = 0; a < 3; ++a) {
    idx[a] = axis_index(p[a], g.d[a], n[a]);
    if (idx[a] < 0 || idx[a] >= n[a]) return true;  // starts outside: escaped
  }
  double t_next[3], t_step[3];
  int step[3];
  for (int a = 0; a < 3; ++a) {
    if (dir[a] > 0.0) {
      step[a] = 1;
      t_next[a] = ((idx[a] + 1) * g.d[a] - p[a]) / dir[a];
      t_step[a] = g.d[a] / dir[a];
    } else if (dir[a] < 0.0) {
      step[a] = -1;
      t_next[a] = (idx[a] * g.d[a] - p[a]) / dir[a];
      t_step[a] = -g.d[a] / dir[a];
    } else {
      step[a] = 0;
      t_next[a] = INFINITY;
      t_step[a] = INFINITY;
    }
  }
  double t = 0.0;
  for (;;) {
    int a = 0;
    if (t_next[1] < t_next[a]) a = 1;
    if (t_next[2] < t_next[a]) a = 2;
    const double t_exit = std::max(t_next[a], t);
    const int64_t v = ((int64_t)idx[2] * g.ny + idx[1]) * g.nx + idx[0];
    if (!visit(v, t, t_exit)) return false;
    t = t_exit;
    idx[a] += step[a];
    if (idx[a] < 0 || idx[a] >= n[a]) return true;
    t_next[a] += t_step[a];
  }
}

// ---- beta+ spectrum and positron range --------------------------------------
// Allowed beta spectrum (Fermi's theory of beta decay): with T the beta
// particle's kinetic energy, E = T + m c^2 its total energy and
// p c = sqrt(T (T + 2 m c^2)),
//   N(T) dT  proportional to  F(Z, E) p E (T_max - T)^2 dT,   0 < T < T_max,
// where F is the non-relativistic Fermi function for a daughter of atomic
// number Z: F = 2 pi eta / (1 - exp(-2 pi eta)) with eta = -sign Z alpha E /
// (p c); sign = +1 for a positron (repulsion: F < 1, vanishing at low T),
// -1 for an electron (attraction: F > 1).
double beta_density(double t, double t_max, int z, int sign) {
  if (!(t > 0.0) || !(t < t_max)) return 0.0;
  const double e = t + kElectronMassMeV;
  const double pc = std::sqrt(t * (t + 2.0 * kElectronMassMeV));
  double f = 1.0;
  if (z != 0) {
    const double x = 2.0 * kPi * (-(double)sign * (double)z * kFineStructure * e / pc);
    f = x / (-std::expm1(-x));
  }
  return f * pc * e * (t_max - t) * (t_max - t);
}

// Sampling of a spectrum of one or more branches (endpoint T_b reached by a
// fraction I_b of the decays): the branch by its share I_b / sum I, then T
// by rejection from that branch's N(T): uniform on (0, T_b), accepted with
// probability N(T) / envelope, the envelope being the branch density's
// maximum over a fine scan raised by 2 % (N is smooth, so the scan is
// within far less).
struct BetaSampler {
  std::vector<double> t_max, env, cum;
  int z = 0, sign = 1;
  BetaSampler(const double* tm, const double* inten, int n, int zz, int sg) : z(zz), sign(sg) {
    constexpr int kScan = 1 << 16;
    double tot = 0.0;
    for (int b = 0; b < n; ++b) tot += inten[b];
    double acc = 0.0;
    for (int b = 0; b < n; ++b) {
      double m = 0.0;
      for (int i = 1; i < kScan; ++i) m = std::max(m, beta_density(tm[b] * i / kScan, tm[b], z, sign));
      t_max.push_back(tm[b]);
      env.push_back(1.02 * m);
      acc += inten[b] / tot;
      cum.push_back(acc);
    }
  }
  double operator()(Rng& r) const {
    size_t b = 0;
    if (cum.size() > 1) {
      const double u = r.u();
      while (b + 1 < cum.size() && u >= cum[b]) ++b;
    }
    for (;;) {
      const double t = r.u() * t_max[b];
      if (r.u() * env[b] < beta_density(t, t_max[b], z, sign)) return t;
    }
  }
};

// Positron range, Katz and Penfold (1952), electrons in low-Z matter:
//   R(T) = 0.412 T^(1.265 - 0.0954 ln T)  g/cm^2,  T in MeV,
// and its inverse: with L = ln T, 0.0954 L^2 - 1.265 L + ln(R / 0.412) = 0,
// the root below L = 1.265 / (2 x 0.0954) (where R increases with T).
double range_kp(double t) {
  if (!(t > 0.0)) return 0.0;
  const double l = std::log(t);
  return 0.412 * std::exp((1.265 - 0.0954 * l) * l);
}

double energy_at_range(double r) {
  if (!(r > 0.0)) return 0.0;
  const double c = std::log(r / 0.412);
  const double disc = 1.265 * 1.265 - 4.0 * 0.0954 * c;
  return std::exp((1.265 - std::sqrt(std::max(disc, 0.0))) / (2.0 * 0.0954));
}

}  // namespace

extern "C" {

// Unnormalised beta+ spectrum N(T) (pinned by the tests through its mean and
// its statistical-shape limit).
double orc_beta_density(double t, double t_max, int32_t z) { return beta_density(t, t_max, z, 1); }

// The same for a positron (sign +1) or an electron (sign -1).
double orc_beta_density_signed(double t, double t_max, int32_t z, int32_t sign) {
  return beta_density(t, t_max, z, sign >= 0 ? 1 : -1);
}

void orc_sample_beta(double t_max, int32_t z, int64_t n, uint64_t seed, double* out) {
  Rng r;
  r.g.seed(seed);
  const double one = 1.0;
  const BetaSampler s(&t_max, &one, 1, z, 1);
  for (int64_t i = 0; i < n; ++i) out[i] = s(r);
}

// Kinetic energies from a spectrum of n_b branches (endpoints, intensities)
// for a positron (sign +1) or an electron (sign -1), as the full simulation
// draws them.
void orc_sample_beta_branches(const double* t_max, const double* intensity, int32_t n_b, int32_t z, int32_t sign,
                              int64_t n, uint64_t seed, double* out) {
  Rng r;
  r.g.seed(seed);
  const BetaSampler s(t_max, intensity, n_b, z, sign >= 0 ? 1 : -1);
  for (int64_t i = 0; i < n; ++i) out[i] = s(r);
}

double orc_range_kp(double t) { return range_kp(t); }
double orc_energy_at_range(double r) { return energy_at_range(r); }

// Path lengths of a ray through the grid (pins the traversal against brute
// force): writes up to cap (voxel, length) pairs, returns the count.
int64_t orc_trace(int32_t nx, int32_t ny, int32_t nz, double dx, double dy, double dz,
                  const double p[3], const double dir[3], int64_t cap, int64_t* voxel,
                  double* length) {
  Grid g{nx, ny, nz, {dx, dy, dz}, nullptr, nullptr};
  int64_t cnt = 0;
  traverse(g, p, dir, [&](int64_t v, double t0, double t1) {
    if (cnt < cap) {
      voxel[cnt] = v;
      length[cnt] = t1 - t0;
    }
    ++cnt;
    return true;
  });
  return cnt;
}

// First-flight distances along a fixed ray through a grid of attenuation
// coefficients mu[v] (1/cm): tau* = -ln u, walk until tau* is used up.  Writes
// the collision distance, or -1 if the photon left the grid.
void orc_first_flight(int32_t nx, int32_t ny, int32_t nz, double dx, double dy, double dz,
                      const double* mu, const double p[3], const double dir[3], int64_t n,
                      uint64_t seed, double* dist) {
  Grid g{nx, ny, nz, {dx, dy, dz}, nullptr, nullptr};
  Rng r;
  r.g.seed(seed);
  for (int64_t i = 0; i < n; ++i) {
    const double tau_star = -std::log(r.u());
    double tau = 0.0, hit = -1.0;
    traverse(g, p, dir, [&](int64_t v, double t0, double t1) {
      const double m = mu[v];
      const double seg = (t1 - t0) * m;
      if (m > 0.0 && tau + seg >= tau_star) {
        hit = t0 + (tau_star - tau) / m;
        return false;
      }
      tau += seg;
      return true;
    });
    dist[i] = hit;
  }
}

void orc_sample_kn_cos(double e_mev, int64_t n, uint64_t seed, double* out) {
  Rng r;
  r.g.seed(seed);
  for (int64_t i = 0; i < n; ++i) out[i] = sample_kn_cos(r, e_mev);
}

void orc_sample_dirs(int64_t n, uint64_t seed, double* out) {
  Rng r;
  r.g.seed(seed);
  for (int64_t i = 0; i < n; ++i) marsaglia(r, out + 3 * i);
}

void orc_rotate(double* d, double c, double phi) { rotate(d, c, phi); }

// Rayleigh cosines as the transport draws them (Thomson shape by rejection).
void orc_sample_thomson_cos(int64_t n, uint64_t seed, double* out) {
  Rng r;
  r.g.seed(seed);
  for (int64_t i = 0; i < n; ++i) out[i] = sample_thomson_cos(r);
}

// n independent real interactions at energy e in material m, density rho,
// with the function the full simulation uses: type[i] (0 Compton, 1
// photoelectric, 2 Rayleigh), the photon energy after it e2[i] and the
// scattering cosine cth[i].
void orc_interactions(const orc_materials* mt, int32_t m, double rho, double e_mev, int64_t n, uint64_t seed,
                      int32_t* type, double* e2, double* cth) {
  Rng r;
  r.g.seed(seed);
  for (int64_t i = 0; i < n; ++i) {
    double phi;
    type[i] = interact(r, mt, m, rho, e_mev, &e2[i], &cth[i], &phi);
  }
}

// ---------------------------------------------------------------------------
// Full simulation.
// ---------------------------------------------------------------------------
typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;            // cm
  const double* density;        // g/cm^3 [nz][ny][nx], x fastest
  const uint8_t* material;      // [V]
  const double* activity;       // [V] >= 0, decay mode only
  const uint8_t* labels;        // [V] 0..n_labels, may be NULL
  int32_t n_labels;
  orc_materials mat;
  int32_t point_mode;           // 1: one photon per history from point[]
  double point[3];              // cm
  double photon_mev;            // 0.511
  double positron_mev;          // 0.25 (decay mode)
  uint64_t n_hist;
  uint64_t first_history;       // history ids continue across runs
  uint64_t seed;
  int32_t batches;              // >= 2
  int32_t threads;              // 0 = all hardware threads
  double activity_bq;           // A(t_s) of Eq. 1
  double beta_max_mev;          // > 0: positron energy from the beta+ spectrum, positron range
  int32_t beta_z;               // daughter's atomic number (Fermi function)
  // Other radionuclides (decay mode).  annihilation: 1 = the positron of every
  // decay gives two back-to-back photons of photon_mev (18F); 0 = none (a
  // beta- emitter).  beta_sign: +1 positron, -1 electron (Fermi function's
  // sign).  n_beta > 0: the spectrum's branches (endpoint, intensity), in
  // place of the single beta_max_mev branch.  Gamma lines: line j is emitted
  // from the decay site with probability gamma_yield[j], independently of
  // the others, in an isotropic direction.
  int32_t annihilation;
  int32_t beta_sign;
  int32_t n_beta;
  const double* beta_endpoint_mev;
  const double* beta_intensity;
  int32_t n_gamma;
  const double* gamma_mev;
  const double* gamma_yield;
} orc_problem;

typedef struct {
  int64_t emitted;     // units
  int64_t deposited;   // units
  int64_t escaped;     // units
  int64_t crossings;   // voxel visits
  int64_t flights;
  int64_t compton, photo, rayleigh, cutoff, escapes;
  int32_t threads_used;
} orc_counters;

int orc_run(const orc_problem* pr, int64_t* tally_sum, double* dose_rate, double* sigma,
            double* organ_mean, double* organ_eps, double* organ_sigma, orc_counters* out_c,
            double* sigma_history) {
  const int64_t V = (int64_t)pr->nx * pr->ny * pr->nz;
  if (V <= 0 || pr->batches < 2 || pr->n_hist < (uint64_t)pr->batches) return 1;
  if (pr->mat.n < 1 || pr->mat.n > 64) return 1;
  for (int64_t v = 0; v < V; ++v)
    if (pr->material[v] >= pr->mat.n || !(pr->density[v] > 0.0)) return 3;
  Grid g{pr->nx, pr->ny, pr->nz, {pr->dx, pr->dy, pr->dz}, pr->density, pr->material};
  const double L[3] = {pr->nx * pr->dx, pr->ny * pr->dy, pr->nz * pr->dz};

  // Decay PDF: linear in the PET value (§2.1); FP64 cumulative table over voxels.
  std::vector<double> cdf;
  if (!pr->point_mode) {
    cdf.resize(V);
    double acc = 0.0;
    for (int64_t v = 0; v < V; ++v) {
      if (!(pr->activity[v] >= 0.0)) return 2;
      acc += pr->activity[v];
      cdf[v] = acc;
    }
    if (!(acc > 0.0)) return 2;
  }

  const int nthreads =
      pr->threads > 0 ? pr->threads : std::max(1u, std::thread::hardware_concurrency());
  const int64_t q_photon = q_units(pr->photon_mev);
  const int64_t q_positron = pr->point_mode ? 0 : q_units(pr->positron_mev);
  const bool beta = !pr->point_mode && (pr->beta_max_mev > 0.0 || pr->n_beta > 0);
  if (beta && pr->n_beta == 0 && !(pr->beta_max_mev < 20.0)) return 1;
  if (pr->n_gamma < 0 || pr->n_gamma > 64 || pr->n_beta < 0 || pr->n_beta > 16) return 1;
  const bool annihilate = pr->annihilation != 0;
  const double one = 1.0, tm1 = beta && pr->n_beta == 0 ? pr->beta_max_mev : 1.0;
  const BetaSampler beta_sampler(pr->n_beta > 0 ? pr->beta_endpoint_mev : &tm1, pr->n_beta > 0 ? pr->beta_intensity : &one,
                                 pr->n_beta > 0 ? pr->n_beta : 1, pr->beta_z, pr->beta_sign < 0 ? -1 : 1);
  const double cut = pr->mat.photon_cut_mev;

  std::vector<int64_t> tb(V);
  std::vector<double> s2(V, 0.0);
  std::fill(tally_sum, tally_sum + V, 0);
  const int nl = pr->n_labels + 1;
  const int B = pr->batches;
  std::vector<double> organ_batch((size_t)B * nl, 0.0);
  std::vector<int64_t> batch_n(B);

  struct Counters {
    int64_t emitted = 0, deposited = 0, escaped = 0, crossings = 0, flights = 0, compton = 0,
            photo = 0, rayleigh = 0, cutoff = 0, escapes = 0;
    std::vector<std::pair<int64_t, int64_t>> hist;   // this history's (voxel, units) so far
  };
  std::vector<Counters> tc(nthreads);
  // History-by-history statistics (Walters et al. 2002): per voxel the sum over
  // histories of the square of each history's total deposit.
  std::vector<double> s2h(sigma_history ? V : 0, 0.0);

  auto deposit = [&](int64_t v, int64_t dq, Counters& c) {
    __atomic_fetch_add(&tb[v], dq, __ATOMIC_RELAXED);
    c.deposited += dq;
    if (sigma_history) {
      bool found = false;
      for (auto& e : c.hist)
        if (e.first == v) { e.second += dq; found = true; break; }
      if (!found) c.hist.emplace_back(v, dq);
    }
  };
  // End of a history: its per-voxel totals enter the sums of squares.
  auto end_history = [&](Counters& c) {
    for (const auto& e : c.hist) {
      const double t2 = (double)e.second * (double)e.second;
      double* slot = &s2h[e.first];
      double old, upd;
      __atomic_load(slot, &old, __ATOMIC_RELAXED);
      do {
        upd = old + t2;
      } while (!__atomic_compare_exchange(slot, &old, &upd, true, __ATOMIC_RELAXED, __ATOMIC_RELAXED));
    }
    c.hist.clear();
  };

  // Transport of one photon from p along dir with energy e0 (§2.1).
  auto transport = [&](Rng& r, const double p0[3], const double d0[3], double e0, Counters& c) {
    double p[3] = {p0[0], p0[1], p0[2]};
    double d[3] = {d0[0], d0[1], d0[2]};
    double e = e0;
    c.emitted += q_units(e0);
    for (;;) {
      // The energy is fixed during a flight: mass attenuation per material once.
      double mass_tot[64];
      for (int m = 0; m < pr->mat.n; ++m) {
        double a, b, cc;
        orc_mass_atten(&pr->mat, m, e, &a, &b, &cc);
        mass_tot[m] = a + b + cc;
      }
      const double tau_star = -std::log(r.u());
      double tau = 0.0, t_hit = -1.0;
      int64_t v_hit = -1;
      ++c.flights;
      const bool escaped = traverse(g, p, d, [&](int64_t v, double t0, double t1) {
        ++c.crossings;
        const double m = pr->density[v] * mass_tot[pr->material[v]];
        const double seg = (t1 - t0) * m;
        if (m > 0.0 && tau + seg >= tau_star) {
          t_hit = t0 + (tau_star - tau) / m;
          v_hit = v;
          return false;
        }
        tau += seg;
        return true;
      });
      if (escaped) {
        c.escaped += q_units(e);
        ++c.escapes;
        return;
      }
      for (int a = 0; a < 3; ++a) p[a] += t_hit * d[a];
      // Keep the collision point inside the collision voxel's grid extent.
      for (int a = 0; a < 3; ++a) p[a] = std::min(std::max(p[a], 0.0), std::nextafter(L[a], 0.0));
      double e2, cth, phi;
      const int type = interact(r, &pr->mat, pr->material[v_hit], pr->density[v_hit], e, &e2, &cth, &phi);
      if (type == kCompton) {
        ++c.compton;
        rotate(d, cth, phi);
        if (e2 < cut) {
          ++c.cutoff;
          deposit(v_hit, q_units(e), c);
          return;
        }
        deposit(v_hit, q_units(e) - q_units(e2), c);
        e = e2;
      } else if (type == kPhoto) {
        ++c.photo;
        deposit(v_hit, q_units(e), c);
        return;
      } else {
        ++c.rayleigh;
        rotate(d, cth, phi);
      }
    }
  };

  // Gamma lines of one decay: each emitted with its yield, from the decay
  // site, in its own isotropic direction.
  auto emit_gammas = [&](Rng& r, const double site[3], Counters& c) {
    for (int j = 0; j < pr->n_gamma; ++j) {
      if (!(r.u() < pr->gamma_yield[j])) continue;
      double dg[3];
      marsaglia(r, dg);
      transport(r, site, dg, pr->gamma_mev[j], c);
    }
  };

  constexpr uint64_t kChunk = 1024;
  uint64_t hist0 = pr->first_history;
  for (int b = 0; b < B; ++b) {
    const uint64_t nb = pr->n_hist / B + ((uint64_t)b < pr->n_hist % B ? 1 : 0);
    batch_n[b] = (int64_t)nb;
    std::fill(tb.begin(), tb.end(), 0);
    // Chunks of histories, each with its own generator seeded from (seed, id of
    // the chunk's first history), so the result does not depend on the number
    // of threads.
    const uint64_t n_chunks = (nb + kChunk - 1) / kChunk;
    std::atomic<uint64_t> next_chunk{0};
    auto worker = [&](int tid) {
      Counters& c = tc[tid];
      Rng r;
      for (;;) {
        const uint64_t ch = next_chunk.fetch_add(1);
        if (ch >= n_chunks) break;
        const uint64_t h_lo = hist0 + ch * kChunk;
        const uint64_t h_hi = std::min(h_lo + kChunk, hist0 + nb);
        std::seed_seq ss{(uint32_t)pr->seed, (uint32_t)(pr->seed >> 32), (uint32_t)h_lo,
                         (uint32_t)(h_lo >> 32)};
        r.g.seed(ss);
        for (uint64_t h = h_lo; h < h_hi; ++h) {
          double p[3], d[3], site[3] = {0.0, 0.0, 0.0};
          int64_t v0 = -1;
          if (pr->point_mode) {
            for (int a = 0; a < 3; ++a) p[a] = pr->point[a];
          } else {
            // Decay voxel by inverse CDF (binary search), position uniform in it.
            const double target = r.u() * cdf[V - 1];
            v0 = std::upper_bound(cdf.begin(), cdf.end(), target) - cdf.begin();
            if (v0 >= V) v0 = V - 1;
            const int64_t ix = v0 % pr->nx, iy = (v0 / pr->nx) % pr->ny,
                          iz = v0 / ((int64_t)pr->nx * pr->ny);
            p[0] = (ix + r.u()) * pr->dx;
            p[1] = (iy + r.u()) * pr->dy;
            p[2] = (iz + r.u()) * pr->dz;
            site[0] = p[0]; site[1] = p[1]; site[2] = p[2];
            if (!beta) {
              // Positron kinetic energy deposited in the decay voxel.
              c.emitted += q_positron;
              deposit(v0, q_positron, c);
            } else {
              // Positron energy from the spectrum; a straight track in an
              // isotropic direction uses up the mass range R(T) voxel by voxel
              // (the continuous-slowing-down energy at the remaining range
              // gives each voxel's deposit); the pair annihilates at its end.
              const double t0 = beta_sampler(r);
              double dp[3];
              marsaglia(r, dp);
              c.emitted += q_units(t0);
              double t_cur = t0, r_rem = range_kp(t0), s_end = 0.0;
              const bool left = traverse(g, p, dp, [&](int64_t v, double a, double b) {
                const double rho = pr->density[v];
                const double m = rho * (b - a);
                if (m >= r_rem) {
                  deposit(v, q_units(t_cur), c);
                  s_end = a + r_rem / rho;
                  return false;
                }
                r_rem -= m;
                const double t_new = energy_at_range(r_rem);
                deposit(v, q_units(t_cur) - q_units(t_new), c);
                t_cur = t_new;
                return true;
              });
              if (left) {
                // the track leaves the grid (vacuum) with what it has left
                // and, for a positron, annihilates outside: both photons escape
                c.escaped += q_units(t_cur);
                if (annihilate) {
                  c.emitted += 2 * q_photon;
                  c.escaped += 2 * q_photon;
                }
                emit_gammas(r, site, c);
                if (sigma_history) end_history(c);
                continue;
              }
              for (int a = 0; a < 3; ++a) p[a] += s_end * dp[a];
            }
          }
          if (pr->point_mode || annihilate) {
            marsaglia(r, d);
            transport(r, p, d, pr->photon_mev, c);
            if (!pr->point_mode) {
              // Annihilation partner: same point, opposite direction (§2.1).
              const double d2[3] = {-d[0], -d[1], -d[2]};
              transport(r, p, d2, pr->photon_mev, c);
            }
          }
          if (!pr->point_mode) emit_gammas(r, site, c);
          if (sigma_history) end_history(c);
        }
      }
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker, t);
    for (auto& t : pool) t.join();

    // Fold the batch: per-decay batch means x_b = T_b / n_b.
    for (int64_t v = 0; v < V; ++v) {
      tally_sum[v] += tb[v];
      const double xb = (double)tb[v] / (double)nb;
      s2[v] += (double)nb * xb * xb;
    }
    if (pr->labels) {
      for (int64_t v = 0; v < V; ++v) {
        const double mass_kg = pr->density[v] * pr->dx * pr->dy * pr->dz * 1e-3;
        const double dose = (double)tb[v] / (double)nb / kUnitsPerMeV * 1e6 * kJoulePerEv / mass_kg;
        organ_batch[(size_t)b * nl + pr->labels[v]] += dose;
      }
    }
    hist0 += nb;
  }

  // Eq. 1: dose rate = D / N_evts * A(t_s); batch sigma of the mean.
  const double N = (double)pr->n_hist;
  std::vector<int64_t> organ_count(nl, 0);
  std::vector<double> osum(nl, 0.0), oeps2(nl, 0.0);
  for (int64_t v = 0; v < V; ++v) {
    const double mass_kg = pr->density[v] * pr->dx * pr->dy * pr->dz * 1e-3;
    const double to_gy = 1e6 * kJoulePerEv / kUnitsPerMeV / mass_kg;  // units -> Gy
    const double mean = (double)tally_sum[v] / N;                       // units per decay
    const double var = std::max(0.0, s2[v] - N * mean * mean) / ((B - 1) * N);
    const double dr = mean * to_gy * pr->activity_bq;
    const double sg = std::sqrt(var) * to_gy * pr->activity_bq;
    if (dose_rate) dose_rate[v] = dr;
    if (sigma) sigma[v] = sg;
    if (sigma_history) {
      // sample variance of the per-history totals, then sigma of their mean
      const double var_h = std::max(0.0, s2h[v] / N - mean * mean) * N / (N - 1.0);
      sigma_history[v] = std::sqrt(var_h / N) * to_gy * pr->activity_bq;
    }
    if (pr->labels) {
      const int l = pr->labels[v];
      organ_count[l] += 1;
      osum[l] += dr;
      const double eps = dr > 0.0 ? sg / dr : 1.0;
      oeps2[l] += eps * eps;
    }
  }
  if (pr->labels) {
    for (int l = 0; l < nl; ++l) {
      const double cnt = (double)organ_count[l];
      // Eq. 2: unweighted mean over the organ's voxels.
      if (organ_mean) organ_mean[l] = cnt > 0 ? osum[l] / cnt : 0.0;
      // Eq. 3: RMS of the voxels' relative uncertainties.
      if (organ_eps) organ_eps[l] = cnt > 0 ? std::sqrt(oeps2[l] / cnt) : 0.0;
      // Batch sigma of the organ mean: m_b = batch organ mean dose per decay,
      // weighted by the batch sizes n_b.
      if (organ_sigma) {
        double mbar = 0.0;
        for (int b = 0; b < B; ++b)
          mbar += batch_n[b] * (organ_batch[(size_t)b * nl + l] / (cnt > 0 ? cnt : 1.0));
        mbar /= N;
        double ss = 0.0;
        for (int b = 0; b < B; ++b) {
          const double mb = organ_batch[(size_t)b * nl + l] / (cnt > 0 ? cnt : 1.0);
          ss += batch_n[b] * (mb - mbar) * (mb - mbar);
        }
        organ_sigma[l] = std::sqrt(ss / ((B - 1) * N)) * pr->activity_bq;
      }
    }
  }
  if (out_c) {
    Counters s;
    for (auto& c : tc) {
      s.emitted += c.emitted; s.deposited += c.deposited; s.escaped += c.escaped;
      s.crossings += c.crossings; s.flights += c.flights; s.compton += c.compton;
      s.photo += c.photo; s.rayleigh += c.rayleigh; s.cutoff += c.cutoff; s.escapes += c.escapes;
    }
    out_c->emitted = s.emitted; out_c->deposited = s.deposited; out_c->escaped = s.escaped;
    out_c->crossings = s.crossings; out_c->flights = s.flights; out_c->compton = s.compton;
    out_c->photo = s.photo; out_c->rayleigh = s.rayleigh; out_c->cutoff = s.cutoff;
    out_c->escapes = s.escapes; out_c->threads_used = nthreads;
  }
  return 0;
}

}  // extern "C"
