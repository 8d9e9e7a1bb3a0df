// Photon transport for ARCHER-NM's method (§2.1): decay sampling, two
// back-to-back 0.511 MeV photons, Woodcock delta tracking through the voxel
// grid, Klein-Nishina Compton (Kahn's sampler), photoelectric absorption,
// optional Rayleigh, 10 keV photon cutoff, int64 fixed-point tally.
//
// One persistent launch per batch.  Each lane owns one photon; a lane whose
// photon ends takes the decay's second photon or, with the rest of its warp,
// refills from a warp-private pool of history ids that one lane grabs from a
// global counter in chunks.  Every iteration of the loop is one flight step
// for every live lane, so lanes stay converged on the flight; the interaction
// work is regrouped (see the `regroup` variant) so that a warp runs Compton
// sampling for a batch of lanes at once instead of once per step.
//
// A history's random numbers come from Philox4x32-10 keyed by the seed with
// counter (block index, stream, history id), so which lane or SM simulates it
// does not matter, and integer atomics make the tally order-independent: a
// fixed seed gives bit-identical tallies.
#include "nm_internal.cuh"

namespace nm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kKahnTrialLimit = 1000;
// Decay-site queue of the single-patient regrouped variant: per warp a ring
// of kQueueCap sampled decays in shared memory, structure of arrays with
// kQueueWords words per decay (site x y z, photon A's direction u v w, the
// two photons' distances to their region boundary, history id lo and hi,
// whether the site lies outside the tracking box).
constexpr int kQueueCap = 64, kQueueWords = 11;

struct Energy {
  float s_c, s_pe, s_r;   // per-unit-density factors: mu/rho = za s_c + zp s_pe + zr s_r
  float inv_mubar;        // 1 / majorant (cm) of the lane's tracking region
};

// Energy-dependent factors, computed once per energy change.  s_c is
// interpolated in ln E from the Klein-Nishina table; the majorant is constant
// over a table bin and taken at the bin's lower edge, which bounds every
// material's mu on the whole bin because all three mu/rho decrease with E.
template <bool RAYLEIGH>
__device__ __forceinline__ Energy energy_factors(float e, const float* __restrict__ kn,
                                                 const float* __restrict__ minv, float ln_lo,
                                                 float inv_dln) {
  Energy f;
  float x = (__logf(e) - ln_lo) * inv_dln;
  x = fminf(fmaxf(x, 0.0f), (float)(kKnTable - 1) - 0x1p-10f);
  const int i = (int)x;
  const float w = x - (float)i;
  const float a = kn[i], b = kn[i + 1];
  f.s_c = fmaf(w, b - a, a);
  const float ie = __fdividef(1.0f, e);
  const float ie2 = ie * ie;
  f.s_pe = ie2 * ie;
  f.s_r = RAYLEIGH ? ie2 : 0.0f;
  f.inv_mubar = minv[i];
  return f;
}

__device__ __forceinline__ uint4 draw(uint32_t& ctr, uint32_t stream, uint32_t hlo, uint32_t hhi,
                                      const PhiloxKey& key) {
  return philox4x32_10(make_uint4(ctr++, stream, hlo, hhi), key);
}

// Kahn's rejection sampler for the Klein-Nishina distribution (Kahn 1954).
// With k = E/m_e c^2, eta = E/E' in [1, 1 + 2k] and x = (eta - 1)/k = 1 - cos θ:
//   branch 1 (prob. (1+2k)/(9+2k)): eta uniform, accept with 4(eta-1)/eta^2;
//   branch 2: eta = (1+2k)/(1+2k r), accept with (cos^2 θ + 1/eta)/2.
// x is formed directly from the uniforms so that cos θ keeps full precision
// at low energy.  One Philox block per trial; its 4th word is the azimuth.
__device__ __forceinline__ float kahn_x(float k, uint32_t& ctr, uint32_t stream, uint32_t hlo,
                                        uint32_t hhi, const PhiloxKey& key, uint32_t& r_phi,
                                        uint32_t& flags) {
  const float two_k = 2.0f * k;
  const float thr = __fdividef(1.0f + two_k, 9.0f + two_k);
  for (int trial = 0;; ++trial) {
    const uint4 r = draw(ctr, stream, hlo, hhi, key);
    const float r1 = u01(r.x), r2 = u01(r.y), r3 = u01(r.z);
    float x;
    bool acc;
    if (r1 <= thr) {
      x = 2.0f * r2;
      const float eta = fmaf(k, x, 1.0f);
      acc = r3 * eta * eta <= 4.0f * k * x;
    } else {
      x = __fdividef(2.0f * (1.0f - r2), fmaf(two_k, r2, 1.0f));
      const float eta = fmaf(k, x, 1.0f);
      const float c = 1.0f - x;
      acc = 2.0f * r3 <= fmaf(c, c, __fdividef(1.0f, eta));
    }
    if (acc || trial + 1 >= kKahnTrialLimit) {
      if (!acc) flags |= NM_DEV_KAHN_LIMIT;
      r_phi = r.w;
      return x;
    }
  }
}

// Klein-Nishina x = 1 - cos(theta) at photon energy e from one uniform word:
// the inverse CDF tabulated (in FP64, on the host) at kKnInvE log-spaced
// energies x kKnInvU + 1 cumulative probabilities, interpolated linearly in
// ln E and in the probability (CDF error below 2e-5 everywhere).  One draw,
// no rejection loop, so the lanes of a warp never wait for each other.
__device__ __forceinline__ float kn_table_x(const TransportParams& p, float e, uint32_t r) {
  float t = (__logf(e) - p.kn_inv_lo) * p.kn_inv_idln;
  t = fminf(fmaxf(t, 0.0f), (float)(kKnInvE - 1) - 0x1p-10f);
  const int i = (int)t;
  const float w = t - (float)i;
  const float sv = u01(r) * (float)kKnInvU;
  const int j = min((int)sv, kKnInvU - 1);
  const float v = sv - (float)j;
  const float* a = p.kn_inv + i * (kKnInvU + 1) + j;
  const float* b = a + (kKnInvU + 1);
  const float a0 = __ldg(a), a1 = __ldg(a + 1), b0 = __ldg(b), b1 = __ldg(b + 1);
  const float x0 = fmaf(v, a1 - a0, a0), x1 = fmaf(v, b1 - b0, b0);
  return fmaf(w, x1 - x0, x0);
}

// New direction at polar cosine c and azimuth phi about (u, v, w).
__device__ __forceinline__ void rotate(float& u, float& v, float& w, float c, float phi) {
  const float s2 = fmaf(-c, c, 1.0f);
  const float s = s2 > 0.0f ? s2 * rsqrtf(s2) : 0.0f;
  float sp, cp;
  __sincosf(phi, &sp, &cp);
  const float t2 = fmaf(-w, w, 1.0f);
  float nu, nv, nw;
  if (t2 > 1e-10f) {
    const float it = rsqrtf(t2);
    const float t = t2 * it;
    nu = fmaf(c, u, s * (u * w * cp - v * sp) * it);
    nv = fmaf(c, v, s * (v * w * cp + u * sp) * it);
    nw = fmaf(c, w, -s * cp * t);
  } else {
    nu = s * cp;
    nv = s * sp;
    nw = w > 0.0f ? c : -c;
  }
  const float n = rsqrtf(fmaf(nu, nu, fmaf(nv, nv, nw * nw)));
  u = nu * n;
  v = nv * n;
  w = nw * n;
}

// Two-region Woodcock tracking.  Inside the tracking box the majorant is the
// grid's; outside it only air-like voxels remain and the majorant is far
// smaller, so a photon leaving the body crosses the surrounding air in one
// step instead of several.  A flight is cut at the box boundary: by the
// memorylessness of the exponential, restarting the flight there with the
// other region's majorant leaves the free-path distribution unchanged.
//
// Slab parameters of the ray (x, y, z) + t (u, v, w), t in cm, against the
// box: it is inside the box for tn < t < tf.
__device__ __forceinline__ void region_slabs(const PatientGeom& G, float x, float y, float z, float u, float v,
                                             float w, float& tn, float& tf) {
  // approximate reciprocals: the box has a one-voxel margin, so a distance
  // off by a few ulp cannot reach a voxel the region's majorant does not cover
  const float iu = __fdividef(1.0f, u * G.inv_dx), iv = __fdividef(1.0f, v * G.inv_dy),
              iw = __fdividef(1.0f, w * G.inv_dz);
  const float ax = (G.blo[0] - x) * iu, bx = (G.bhi[0] - x) * iu;
  const float ay = (G.blo[1] - y) * iv, by = (G.bhi[1] - y) * iv;
  const float az = (G.blo[2] - z) * iw, bz = (G.bhi[2] - z) * iw;
  // fminf/fmaxf drop the NaN of 0 * inf (a ray in a box face, parallel to it)
  tf = fminf(fmaxf(ax, bx), fminf(fmaxf(ay, by), fmaxf(az, bz)));
  tn = fmaxf(fminf(ax, bx), fmaxf(fminf(ay, by), fminf(az, bz)));
}

constexpr float kInf = __builtin_huge_valf();

// Distance (cm) from (x, y, z) along (u, v, w) to the boundary of the lane's
// region: from inside, to the box's far side; from outside, to its near side,
// or +inf when the ray misses the box (a ray that has left the convex box
// never meets it again).
__device__ __forceinline__ float region_distance(const PatientGeom& G, bool out, float x, float y, float z,
                                                 float u, float v, float w) {
  float tn, tf;
  region_slabs(G, x, y, z, u, v, w, tn, tf);
  if (!out) return tf;
  return tn <= tf && tf > 0.0f ? fmaxf(tn, 0.0f) : kInf;
}

// The same for the ray and for its reverse (photon B leaves the decay site
// opposite to photon A): reversing the ray maps (tn, tf) to (-tf, -tn).
__device__ __forceinline__ void region_distance_pair(const PatientGeom& G, bool out, float x, float y, float z,
                                                     float u, float v, float w, float& fwd, float& rev) {
  float tn, tf;
  region_slabs(G, x, y, z, u, v, w, tn, tf);
  if (!out) {
    fwd = tf;
    rev = -tn;
  } else {
    fwd = tn <= tf && tf > 0.0f ? fmaxf(tn, 0.0f) : kInf;
    rev = tn <= tf && tn < 0.0f ? fmaxf(-tf, 0.0f) : kInf;
  }
}

__device__ __forceinline__ bool outside_box(const PatientGeom& G, float x, float y, float z) {
  return !(x >= G.blo[0] && x < G.bhi[0] && y >= G.blo[1] && y < G.bhi[1] && z >= G.blo[2] && z < G.bhi[2]);
}

// 1 / majorant at energy e from a region's table (same bin as energy_factors).
__device__ __forceinline__ float inv_majorant_at(float e, const float* __restrict__ minv, float ln_lo,
                                                 float inv_dln) {
  float x = (__logf(e) - ln_lo) * inv_dln;
  x = fminf(fmaxf(x, 0.0f), (float)(kKnTable - 1) - 0x1p-10f);
  return minv[(int)x];
}

// Decay site and first-photon direction of history (hlo, hhi).
struct Site {
  int v;              // decay voxel (-1 in point mode)
  float x, y, z;      // voxel units
  float u, v_, w;     // direction of photon A
};

__device__ __forceinline__ Site sample_site(const PatientGeom& G, const PhiloxKey& key,
                                           uint32_t hlo, uint32_t hhi) {
  Site s;
  uint32_t ctr = 0;
  uint4 r = draw(ctr, kStreamSource, hlo, hhi, key);
  uint32_t rc, rphi;
  if (G.source_mode == NM_SOURCE_DECAY) {
    // Alias table: 64 random bits pick a column uniformly, one more the side.
    const uint64_t r64 = ((uint64_t)r.y << 32) | r.x;
    const uint64_t col = __umul64hi(r64, G.n_active);
    const uint4 a = __ldg(G.alias + col);
    s.v = (u01(r.z) < __uint_as_float(a.x)) ? (int)a.y : (int)a.z;
    const int nxy = G.nx * G.ny;
    const int iz = s.v / nxy;
    const int rem = s.v - iz * nxy;
    const int iy = rem / G.nx;
    const int ix = rem - iy * G.nx;
    const uint32_t rx = r.w;
    r = draw(ctr, kStreamSource, hlo, hhi, key);
    // Uniform inside the voxel; keep ix + u below ix + 1 after rounding.
    s.x = fminf((float)ix + u01(rx), __int_as_float(__float_as_int((float)(ix + 1)) - 1));
    s.y = fminf((float)iy + u01(r.x), __int_as_float(__float_as_int((float)(iy + 1)) - 1));
    s.z = fminf((float)iz + u01(r.y), __int_as_float(__float_as_int((float)(iz + 1)) - 1));
    rc = r.z;
    rphi = r.w;
  } else {
    s.v = -1;
    s.x = G.px;
    s.y = G.py;
    s.z = G.pz;
    rc = r.x;
    rphi = r.y;
  }
  // Isotropic: cos θ uniform on (-1, 1), azimuth uniform.
  const float c = fmaf(2.0f, u01(rc), -1.0f);
  const float sn = sqrtf(fmaxf(0.0f, fmaf(-c, c, 1.0f)));
  float sp, cp;
  __sincosf(fmaf(kTwoPi, u01(rphi), -3.14159265f), &sp, &cp);
  s.u = sn * cp;
  s.v_ = sn * sp;
  s.w = c;
  return s;
}

// Katz-Penfold range of a positron of kinetic energy t (MeV), g/cm^2:
// R = 0.412 t^(1.265 - 0.0954 ln t); and its inverse, the lower root of
// 0.0954 L^2 - 1.265 L + ln(R / 0.412) = 0 in L = ln t.
__device__ __forceinline__ float kp_range(float t) {
  const float l = logf(t);
  return 0.412f * expf((1.265f - 0.0954f * l) * l);
}
__device__ __forceinline__ float kp_energy(float r) {
  if (!(r > 0.0f)) return 0.0f;
  const float c = logf(r * (1.0f / 0.412f));
  const float disc = fmaxf(fmaf(-4.0f * 0.0954f, c, 1.265f * 1.265f), 0.0f);
  return expf((1.265f - sqrtf(disc)) * (1.0f / (2.0f * 0.0954f)));
}

// Positron kinetic energy (MeV) for the uniform word r: linear interpolation
// in the inverse-CDF table of the beta+ spectrum.
__device__ __forceinline__ float beta_energy(const float* __restrict__ tab, uint32_t r) {
  const float sv = u01(r) * (float)kBetaTable;
  const int i = min((int)sv, kBetaTable - 1);
  const float ta = __ldg(tab + i), tb = __ldg(tab + i + 1);
  return fmaf(sv - (float)i, tb - ta, ta);
}

// The positron of a decay, beta+ spectrum mode: kinetic energy from the
// inverse-CDF table (linear between nodes), an isotropic straight track from
// the decay site (x, y, z, voxel units; in voxel v0) walked voxel by voxel,
// each voxel using up rho x (path in it) of the mass range and keeping the
// energy lost there, q(T before) - q(T at the range left), until the range
// is spent.  On return (x, y, z) is the end of the track, where the pair
// annihilates, and q0 the positron's energy in tally units.  Returns false if
// the track left the grid; q_left is then the energy it carried out.
template <class Dep>
__device__ __forceinline__ bool positron_track(const PatientGeom& G, const PhiloxKey& key, uint32_t hlo,
                                               uint32_t hhi, int v0, float& x, float& y, float& z,
                                               uint32_t& q0, uint32_t& q_left, Dep&& dep) {
  uint32_t ctr = 0;
  const uint4 r = draw(ctr, kStreamPositron, hlo, hhi, key);
  const float t0 = beta_energy(G.beta_tab, r.x);
  q0 = (uint32_t)q_units(t0);
  const float cz = fmaf(2.0f, u01(r.y), -1.0f);
  const float sn = sqrtf(fmaxf(0.0f, fmaf(-cz, cz, 1.0f)));
  float sp, cp;
  __sincosf(fmaf(kTwoPi, u01(r.z), -3.14159265f), &sp, &cp);
  const float ux = sn * cp, uy = sn * sp, uz = cz;
  const int nxy = G.nx * G.ny;
  int iz = v0 / nxy;
  int iy = (v0 - iz * nxy) / G.nx;
  int ix = v0 - iz * nxy - iy * G.nx;
  // per axis: track length (cm) to the next voxel plane and between planes
  const float dx = 1.0f / G.inv_dx, dy = 1.0f / G.inv_dy, dz = 1.0f / G.inv_dz;
  const int sx = ux > 0.0f ? 1 : -1, sy = uy > 0.0f ? 1 : -1, sz = uz > 0.0f ? 1 : -1;
  float tnx = ux != 0.0f ? ((float)(ix + (ux > 0.0f)) - x) * dx / ux : kInf;
  float tny = uy != 0.0f ? ((float)(iy + (uy > 0.0f)) - y) * dy / uy : kInf;
  float tnz = uz != 0.0f ? ((float)(iz + (uz > 0.0f)) - z) * dz / uz : kInf;
  const float dtx = ux != 0.0f ? dx / fabsf(ux) : kInf;
  const float dty = uy != 0.0f ? dy / fabsf(uy) : kInf;
  const float dtz = uz != 0.0f ? dz / fabsf(uz) : kInf;
  float r_left = kp_range(t0), tcur = 0.0f;
  uint32_t q_cur = q0;
  int v = v0;
  // a straight line crosses at most nx + ny + nz voxels
  const int limit = G.nx + G.ny + G.nz + 2;
  for (int it = 0;; ++it) {
    const bool bx = tnx <= tny && tnx <= tnz;
    const bool by = !bx && tny <= tnz;
    const float tn = bx ? tnx : by ? tny : tnz;
    const float rho = __uint_as_float(__ldg(G.vox + v) & ~7u);
    const float seg = fmaxf(tn - tcur, 0.0f);
    if (rho * seg >= r_left || it + 1 >= limit) {
      // the range ends in this voxel: it keeps the rest of the energy
      if (q_cur) dep(v, q_cur);
      const float send = tcur + fminf(r_left / rho, seg);
      x = fminf(fmaxf(fmaf(send * G.inv_dx, ux, x), (float)ix), __int_as_float(__float_as_int((float)(ix + 1)) - 1));
      y = fminf(fmaxf(fmaf(send * G.inv_dy, uy, y), (float)iy), __int_as_float(__float_as_int((float)(iy + 1)) - 1));
      z = fminf(fmaxf(fmaf(send * G.inv_dz, uz, z), (float)iz), __int_as_float(__float_as_int((float)(iz + 1)) - 1));
      return true;
    }
    r_left -= rho * seg;
    const uint32_t q_new = min((uint32_t)q_units(kp_energy(r_left)), q_cur);
    if (q_cur > q_new) dep(v, q_cur - q_new);
    q_cur = q_new;
    tcur = tn;
    bool left;
    if (bx) {
      ix += sx; v += sx; tnx += dtx; left = (unsigned)ix >= (unsigned)G.nx;
    } else if (by) {
      iy += sy; v += sy * G.nx; tny += dty; left = (unsigned)iy >= (unsigned)G.ny;
    } else {
      iz += sz; v += sz * nxy; tnz += dtz; left = (unsigned)iz >= (unsigned)G.nz;
    }
    if (left) {
      q_left = q_cur;
      return false;
    }
  }
}

// Adds dq units to *cell.  With WARP_AGG the lanes that hit the same cell
// (same address, so lanes of different patients never merge) add their
// deposits with one warp reduction and one atomic.
template <bool WARP_AGG>
__device__ __forceinline__ void tally_flush(ull* cell, bool has, uint32_t dq, uint32_t lane) {
  if (WARP_AGG) {
    const unsigned m = __ballot_sync(kFull, has);
    if (has) {
      const unsigned g = __match_any_sync(m, (unsigned long long)cell);
      const unsigned sum = __reduce_add_sync(g, dq);
      if (lane == (unsigned)(__ffs(g) - 1)) atomicAdd(cell, (ull)sum);
    }
  } else if (has) {
    atomicAdd(cell, (ull)dq);
  }
}

__device__ __forceinline__ ull warp_sum(ull x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Compton event at energy e: Kahn-sampled angle, new energy and direction, and
// the local deposit (the electron's energy, or everything below the cutoff).
template <bool RAYLEIGH>
// With the tabulated sampler the angle takes the two words (rk, rp) that
// the flight step which found the event drew but did not use; Kahn's sampler
// draws its own blocks.
__device__ __forceinline__ void compton(const TransportParams& p, const float* s_kn,
                                        const float* s_minv, float& e, int32_t& qe, Energy& f,
                                        float& ux, float& uy, float& uz, uint32_t& ctr,
                                        uint32_t stream, uint32_t hlo, uint32_t hhi,
                                        bool& alive, uint32_t& dq, uint32_t& flags,
                                        unsigned long long* s_cnt, uint32_t rk, uint32_t rp) {
  uint32_t rphi;
  const float k = e * kInvElectronMassMeV;
  float x;
  if (p.kn_inv) {
    x = kn_table_x(p, e, rk);
    rphi = rp;
  } else {
    x = kahn_x(k, ctr, stream, hlo, hhi, p.key, rphi, flags);
  }
  const float e2 = __fdividef(e, fmaf(k, x, 1.0f));
  rotate(ux, uy, uz, 1.0f - x, fmaf(kTwoPi, u01(rphi), -3.14159265f));
  if (e2 < p.cut) {
    dq = (uint32_t)qe;
    alive = false;
    atomicAdd(&s_cnt[kCtrCutoff], 1ull);
  } else {
    const int32_t q2 = q_units(e2);
    dq = (uint32_t)(qe - q2);
    e = e2;
    qe = q2;
    f = energy_factors<RAYLEIGH>(e, s_kn, s_minv, p.ln_e_lo, p.inv_dln_e);
  }
}

// History statistics: a lane lists its current history's deposits per voxel
// (kHistVoxels entries in shared memory, structure of arrays over the CTA) and
// adds them to the tally, with their squares to the 128-bit sums, when the
// history ends (the lane takes its next history, or the kernel ends).
struct HistList {
  uint32_t* v;   // voxel of entry i at v[i * stride]
  uint32_t* q;   // units
  int stride;
};

__device__ __forceinline__ void hist_flush(const HistList& L, int& n, ull* tally, ull* lo, ull* hi) {
  for (int i = 0; i < n; ++i) {
    const uint32_t v = L.v[i * L.stride], t = L.q[i * L.stride];
    atomicAdd(tally + v, (ull)t);
    const ull t2 = (ull)t * t;
    const ull old = atomicAdd(lo + v, t2);
    if (old + t2 < old) atomicAdd(hi + v, 1ull);   // carry into the high word
  }
  n = 0;
}

__device__ __forceinline__ void hist_add(const HistList& L, int& n, uint32_t v, uint32_t dq, ull* tally, ull* lo,
                                         ull* hi, ull* splits) {
  for (int i = 0; i < n; ++i)
    if (L.v[i * L.stride] == v) {
      L.q[i * L.stride] += dq;
      return;
    }
  if (n == kHistVoxels) {
    // more voxels than a lane keeps: the totals so far are squared now
    hist_flush(L, n, tally, lo, hi);
    atomicAdd(splits, 1ull);
  }
  L.v[n * L.stride] = v;
  L.q[n * L.stride] = dq;
  ++n;
}

template <bool WARP_AGG, bool RAYLEIGH, bool REGROUP, bool MULTI, bool HIST, bool BETA>
__global__ void __launch_bounds__(512, 2) transport_kernel(const TransportParams p) {
  static_assert(!HIST || (!WARP_AGG && !MULTI), "history statistics: one patient, lane-wise deposits");
  static_assert(!BETA || (!WARP_AGG && !MULTI), "beta+ spectrum: one patient, lane-wise deposits");
  __shared__ float s_kn[kKnTable];
  __shared__ float s_minv[kKnTable];
  __shared__ float s_minv_out[kKnTable];
  __shared__ MaterialCoef s_mat[NM_MAX_MATERIALS];
  __shared__ Energy s_f0;
  __shared__ float s_inv0_out;              // 1 / majorant outside the box at e0
  // Per patient, indexed by CounterSlot: the rare events (photo, cutoff,
  // rayleigh, killed units) counted here directly, and (multi) the lanes'
  // register counters handed over when a lane changes patient.
  __shared__ unsigned long long s_cnt[MULTI ? kMaxBatchPatients : 1][10];  // [8]: positron, [9]: gamma units
  __shared__ PatientGeom s_geom[MULTI ? kMaxBatchPatients : 1];
  extern __shared__ float s_site[];         // [9][blockDim]: decay site, photon A direction, photon B's
                                            // distance to its region boundary, a pending Compton's two words;
                                            // then the history lists (HIST) and the gamma origin (BETA)
  const int n_pat = MULTI ? p.n_patients : 1;
  for (int i = threadIdx.x; i < kKnTable; i += blockDim.x) {
    s_kn[i] = p.kn[i];
    s_minv[i] = p.minv[i];
    s_minv_out[i] = p.minv_out[i];
  }
  if (threadIdx.x < NM_MAX_MATERIALS) s_mat[threadIdx.x] = p.mat[threadIdx.x];
  for (int i = threadIdx.x; i < n_pat * 10; i += blockDim.x) s_cnt[i / 10][i % 10] = 0;
  if (MULTI)
    for (int i = threadIdx.x; i < n_pat; i += blockDim.x) s_geom[i] = p.patients[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    s_f0 = energy_factors<RAYLEIGH>(p.e0, s_kn, s_minv, p.ln_e_lo, p.inv_dln_e);
    s_inv0_out = inv_majorant_at(p.e0, s_minv_out, p.ln_e_lo, p.inv_dln_e);
  }
  __syncthreads();
  float* site = s_site + threadIdx.x;
  const int nb = blockDim.x;
  const HistList hl{reinterpret_cast<uint32_t*>(s_site + 9 * nb) + threadIdx.x,
                    reinterpret_cast<uint32_t*>(s_site + (9 + kHistVoxels) * nb) + threadIdx.x, nb};
  int hn = 0;                            // entries in this lane's history list
  // nuclide variant: the decay site (origin of the gamma lines) and the lines
  // of this decay still to be emitted
  float* gsite = s_site + (9 + (HIST ? 2 * kHistVoxels : 0)) * nb + threadIdx.x;
  uint32_t gmask = 0;

  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt_mask = (1u << lane) - 1u;
  // Warp-uniform work pool [pool_next, pool_end) of patient wp; the warps start
  // spread over the patients.
  uint32_t pool_next = 0, pool_end = 0;
  int wp = MULTI ? (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % n_pat) : 0;
  int pi = 0;                            // this lane's patient
  int cpi = 0;                           // patient the lane's counters belong to
  bool done = false, alive = false, pending_b = false, pending_c = false;
  float px = 0.f, py = 0.f, pz = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
  float e = 0.f;
  Energy f = s_f0;
  int32_t qe = 0;
  int cv = 0;                            // voxel of a pending Compton event
  uint32_t hlo = 0, hhi = 0, stream = 0, ctr = 0;
  bool out = false;                      // outside the tracking box
  float rem = 0.f;                       // cm to the region boundary along (ux, uy, uz)
  int steps = 0;
  uint32_t n_steps = 0, n_compton = 0, n_esc = 0, flags = 0;
  ull escaped = 0;

  // The single-patient regrouped variant samples decays ahead of need: the
  // whole warp fills its site queue 32 decays at a time, and a lane whose
  // photons have ended takes the next queued decay at once, so no lane waits
  // for a refill pass and the sampling runs with every lane busy.
  constexpr bool SITEQ = REGROUP && !MULTI && !HIST && !BETA;
  float* const q_base = s_site + 9 * nb + (threadIdx.x >> 5) * (kQueueCap * kQueueWords);
  uint32_t q_head = 0, q_count = 0;      // warp-uniform ring state
  bool drained = false;                  // warp-uniform: every history id has been handed out

  for (;;) {
    if constexpr (SITEQ) {
      // ---- fill the site queue: one new decay per lane -----------------------
      if (q_count < 32 && !drained) {
        const uint32_t avail = pool_end - pool_next;
        uint32_t fresh = 0, fresh_end = 0;
        if (avail < 32) {
          if (lane == 0) {
            const unsigned f0 = atomicAdd(p.g.work, (unsigned)p.chunk);
            if ((uint64_t)f0 < p.g.n_hist) {
              fresh = f0;
              fresh_end = (uint32_t)min((uint64_t)f0 + (uint64_t)p.chunk, p.g.n_hist);
            }
          }
          fresh = __shfl_sync(kFull, fresh, 0);
          fresh_end = __shfl_sync(kFull, fresh_end, 0);
        }
        uint32_t idx = 0;
        bool got = true;
        if (lane < avail) {
          idx = pool_next + lane;
        } else if (fresh + (lane - avail) < fresh_end) {
          idx = fresh + (lane - avail);
        } else {
          got = false;
        }
        if (avail < 32) {
          pool_next = min(fresh + (32u - avail), fresh_end);
          pool_end = fresh_end;
          drained = fresh_end == 0;
        } else {
          pool_next += 32;
        }
        const uint32_t n_got = __popc(__ballot_sync(kFull, got));   // lanes 0 .. n_got - 1
        bool has = false;
        ull* cell = nullptr;
        if (got) {
          const uint64_t h = p.g.hist_begin + idx;
          const uint32_t slo = (uint32_t)h, shi = (uint32_t)(h >> 32);
          const Site st = sample_site(p.g, p.key, slo, shi);
          const bool o = outside_box(p.g, st.x, st.y, st.z);
          float ra, rb;
          region_distance_pair(p.g, o, st.x, st.y, st.z, st.u, st.v_, st.w, ra, rb);
          float* qs = q_base + ((q_head + q_count + lane) & (kQueueCap - 1));
          uint32_t* qw = reinterpret_cast<uint32_t*>(qs);
          qs[0] = st.x; qs[kQueueCap] = st.y; qs[2 * kQueueCap] = st.z;
          qs[3 * kQueueCap] = st.u; qs[4 * kQueueCap] = st.v_; qs[5 * kQueueCap] = st.w;
          qs[6 * kQueueCap] = ra; qs[7 * kQueueCap] = rb;
          qw[8 * kQueueCap] = slo; qw[9 * kQueueCap] = shi; qw[10 * kQueueCap] = o ? 1u : 0u;
          if (p.g.source_mode == NM_SOURCE_DECAY) {
            has = p.g.q_positron > 0;
            cell = p.g.tally + st.v;
          }
        }
        tally_flush<WARP_AGG>(cell, has, (uint32_t)p.g.q_positron, lane);
        q_count += n_got;
        __syncwarp();
      }
      // ---- lanes without a photon: the decay's second one, or the next decay -
      const unsigned want = __ballot_sync(kFull, !alive && !pending_b);
      const uint32_t n_pop = min((uint32_t)__popc(want), q_count);
      if (!alive) {
        if (pending_b) {
          pending_b = false;
          alive = true;
          px = site[0]; py = site[nb]; pz = site[2 * nb];
          ux = -site[3 * nb]; uy = -site[4 * nb]; uz = -site[5 * nb];
          e = p.e0; qe = p.q_e0; f = s_f0;
          stream = kStreamPhotonB; ctr = 0; steps = 0;
          out = outside_box(p.g, px, py, pz);
          rem = site[6 * nb];
          if (out) f.inv_mubar = s_inv0_out;
        } else {
          const uint32_t rank = __popc(want & lt_mask);
          if (rank < n_pop) {
            const float* qs = q_base + ((q_head + rank) & (kQueueCap - 1));
            const uint32_t* qw = reinterpret_cast<const uint32_t*>(qs);
            px = qs[0]; py = qs[kQueueCap]; pz = qs[2 * kQueueCap];
            ux = qs[3 * kQueueCap]; uy = qs[4 * kQueueCap]; uz = qs[5 * kQueueCap];
            rem = qs[6 * kQueueCap];
            hlo = qw[8 * kQueueCap]; hhi = qw[9 * kQueueCap];
            out = qw[10 * kQueueCap] != 0u;
            e = p.e0; qe = p.q_e0; f = s_f0;
            if (out) f.inv_mubar = s_inv0_out;
            stream = kStreamPhotonA; ctr = 0; steps = 0;
            alive = true;
            if (p.g.source_mode == NM_SOURCE_DECAY) {
              site[0] = px; site[nb] = py; site[2 * nb] = pz;
              site[3 * nb] = ux; site[4 * nb] = uy; site[5 * nb] = uz;
              site[6 * nb] = qs[7 * kQueueCap];
              pending_b = true;
            }
          }
        }
      }
      q_head = (q_head + n_pop) & (kQueueCap - 1);
      q_count -= n_pop;
      __syncwarp();
      if (!__any_sync(kFull, alive) && q_count == 0 && drained) break;
    } else {
    // ---- second photon of the decay: same site, opposite direction ----------
    if (!alive && pending_b) {
      pending_b = false;
      alive = true;
      px = site[0]; py = site[nb]; pz = site[2 * nb];
      ux = -site[3 * nb]; uy = -site[4 * nb]; uz = -site[5 * nb];
      e = p.e0; qe = p.q_e0; f = s_f0;
      stream = kStreamPhotonB; ctr = 0; steps = 0;
      const PatientGeom& GB = MULTI ? s_geom[pi] : p.g;
      out = outside_box(GB, px, py, pz);
      rem = site[6 * nb];
      if (out) f.inv_mubar = s_inv0_out;
    } else if (BETA && !alive && gmask) {
      // ---- next gamma line of the decay: from the decay site, isotropic ------
      const int j = __ffs(gmask) - 1;
      gmask &= gmask - 1;
      alive = true;
      px = gsite[0]; py = gsite[nb]; pz = gsite[2 * nb];
      stream = kStreamGamma0 + (uint32_t)j; ctr = 0; steps = 0;
      const uint4 rd = draw(ctr, stream, hlo, hhi, p.key);
      const float c = fmaf(2.0f, u01(rd.x), -1.0f);
      const float sn = sqrtf(fmaxf(0.0f, fmaf(-c, c, 1.0f)));
      float sp, cp;
      __sincosf(fmaf(kTwoPi, u01(rd.y), -3.14159265f), &sp, &cp);
      ux = sn * cp; uy = sn * sp; uz = c;
      e = p.gamma_e[j]; qe = p.gamma_q[j];
      atomicAdd(&s_cnt[0][9], (ull)(uint32_t)qe);
      out = outside_box(p.g, px, py, pz);
      f = energy_factors<RAYLEIGH>(e, s_kn, out ? s_minv_out : s_minv, p.ln_e_lo, p.inv_dln_e);
      rem = region_distance(p.g, out, px, py, pz, ux, uy, uz);
    }
    // ---- refill: lanes without a photon take new histories from the pool ----
    const unsigned need = __ballot_sync(kFull, !alive && !done);
    bool refill = need != 0;
    if (REGROUP && refill) {
      // Start new histories for many lanes at once, once enough lanes wait or
      // nothing else can fly.
      const unsigned flying = __ballot_sync(kFull, alive && !pending_c);
      refill = __popc(need) >= (unsigned)p.regroup_refill || flying == 0;
    }
    if (refill) {
      const uint32_t cnt = __popc(need);
      const uint32_t avail = pool_end - pool_next;
      uint32_t fresh = 0, fresh_end = 0;
      int nwp = wp;
      if (avail < cnt) {
        // Grab a chunk from the current patient's queue; a drained queue moves
        // the warp on to the next patient.
        if (lane == 0) {
          for (int t = 0; t < n_pat; ++t) {
            const PatientGeom& Q = MULTI ? s_geom[nwp] : p.g;
            const unsigned f0 = atomicAdd(Q.work, (unsigned)p.chunk);
            if ((uint64_t)f0 < Q.n_hist) {
              fresh = f0;
              fresh_end = (uint32_t)min((uint64_t)f0 + (uint64_t)p.chunk, Q.n_hist);
              break;
            }
            if (MULTI) nwp = nwp + 1 < n_pat ? nwp + 1 : 0;
          }
        }
        fresh = __shfl_sync(kFull, fresh, 0);
        fresh_end = __shfl_sync(kFull, fresh_end, 0);
        nwp = __shfl_sync(kFull, nwp, 0);
      }
      bool has = false;
      ull* cell = nullptr;
      if (!alive && !done) {
        const uint32_t rank = __popc(need & lt_mask);
        uint32_t idx = 0;
        bool got = true;
        int npi = wp;
        if (rank < avail) {
          idx = pool_next + rank;
        } else if (fresh + (rank - avail) < fresh_end) {
          idx = fresh + (rank - avail);
          npi = nwp;
        } else {
          got = false;
          if (fresh_end == 0) done = true;   // every queue is drained
        }
        if (got) {
          if (MULTI && npi != cpi) {
            // counters belong to one patient: hand them over before switching
            atomicAdd(&s_cnt[cpi][kCtrSteps], (ull)n_steps);
            atomicAdd(&s_cnt[cpi][kCtrCompton], (ull)n_compton);
            atomicAdd(&s_cnt[cpi][kCtrEscapes], (ull)n_esc);
            atomicAdd(&s_cnt[cpi][kCtrEscapedUnits], escaped);
            n_steps = n_compton = n_esc = 0;
            escaped = 0;
            cpi = npi;
          }
          pi = npi;
          if (HIST && hn) hist_flush(hl, hn, p.g.tally, p.s2h_lo, p.s2h_hi);   // the previous history ends
          const PatientGeom& G = MULTI ? s_geom[pi] : p.g;
          const uint64_t h = G.hist_begin + idx;
          hlo = (uint32_t)h;
          hhi = (uint32_t)(h >> 32);
          Site st = sample_site(G, p.key, hlo, hhi);
          bool pair = true;                  // the annihilation photons start inside the grid
          if (BETA && G.source_mode == NM_SOURCE_DECAY) {
            // another radionuclide: gamma lines of this decay, emitted later
            // from the decay site (the nucleus), one photon at a time
            gsite[0] = st.x; gsite[nb] = st.y; gsite[2 * nb] = st.z;
            uint32_t m = 0, gc = 0;
            for (int j0 = 0; j0 < p.n_gamma; j0 += 4) {
              const uint4 rg = draw(gc, kStreamGammaSelect, hlo, hhi, p.key);
              const uint32_t w4[4] = {rg.x, rg.y, rg.z, rg.w};
              for (int k = 0; k < 4 && j0 + k < p.n_gamma; ++k)
                if (u01(w4[k]) < p.gamma_y[j0 + k]) m |= 1u << (j0 + k);
            }
            gmask = m;
          }
          if (BETA && G.beta_tab) {
            uint32_t q0 = 0, q_left = 0;
            pair = positron_track(G, p.key, hlo, hhi, st.v, st.x, st.y, st.z, q0, q_left,
                                  [&](int v, uint32_t dq) {
                                    if (HIST)
                                      hist_add(hl, hn, (uint32_t)v, dq, p.g.tally, p.s2h_lo, p.s2h_hi,
                                               p.g.counters + kCtrHistSplits);
                                    else
                                      atomicAdd(G.tally + v, (ull)dq);
                                  });
            atomicAdd(&s_cnt[MULTI ? pi : 0][8], (ull)q0);
            if (!pair) escaped += (ull)q_left + (p.annihilate ? 2ull * (ull)(uint32_t)p.q_e0 : 0ull);
          }
          if (BETA && G.source_mode == NM_SOURCE_DECAY && G.q_positron > 0 && !p.annihilate) {
            // no annihilation photon to carry the local deposit: tally it here
            if (HIST)
              hist_add(hl, hn, (uint32_t)st.v, (uint32_t)G.q_positron, p.g.tally, p.s2h_lo, p.s2h_hi,
                       p.g.counters + kCtrHistSplits);
            else
              atomicAdd(G.tally + st.v, (ull)(uint32_t)G.q_positron);
          }
          if (BETA && !p.annihilate && G.source_mode == NM_SOURCE_DECAY) pair = false;
          if (pair) {
          px = st.x; py = st.y; pz = st.z;
          ux = st.u; uy = st.v_; uz = st.w;
          e = p.e0; qe = p.q_e0; f = s_f0;
          stream = kStreamPhotonA; ctr = 0; steps = 0;
          alive = true;
          out = outside_box(G, px, py, pz);
          if (out) f.inv_mubar = s_inv0_out;
          float rem_b;
          region_distance_pair(G, out, px, py, pz, ux, uy, uz, rem, rem_b);
          if (G.source_mode == NM_SOURCE_DECAY) {
            site[0] = st.x; site[nb] = st.y; site[2 * nb] = st.z;
            site[3 * nb] = st.u; site[4 * nb] = st.v_; site[5 * nb] = st.w;
            site[6 * nb] = rem_b;
            pending_b = true;
            if (HIST) {
              if (G.q_positron > 0)
                hist_add(hl, hn, (uint32_t)st.v, (uint32_t)G.q_positron, p.g.tally, p.s2h_lo, p.s2h_hi,
                         p.g.counters + kCtrHistSplits);
            } else {
              has = G.q_positron > 0;
              cell = G.tally + st.v;
            }
          }
          }
        }
      }
      if (avail < cnt) {
        pool_next = min(fresh + (cnt - avail), fresh_end);
        pool_end = fresh_end;
        wp = nwp;
      } else {
        pool_next += cnt;
      }
      tally_flush<WARP_AGG>(cell, has, (uint32_t)(MULTI ? s_geom[pi].q_positron : p.g.q_positron), lane);
    }
    if (!__any_sync(kFull, alive || !done)) break;
    }

    const PatientGeom& G = MULTI ? s_geom[pi] : p.g;
    bool has = false;
    int dv = 0;
    uint32_t dq = 0;
    // ---- Compton passes (regrouped: run when enough lanes wait) -------------
    if (REGROUP) {
      const unsigned waiting = __ballot_sync(kFull, pending_c);
      const unsigned flying = __ballot_sync(kFull, alive && !pending_c);
      if (waiting && (__popc(waiting) >= (unsigned)p.regroup_compton || flying == 0)) {
        if (pending_c) {
          pending_c = false;
          const uint32_t* words = reinterpret_cast<const uint32_t*>(site);
          compton<RAYLEIGH>(p, s_kn, out ? s_minv_out : s_minv, e, qe, f, ux, uy, uz, ctr, stream, hlo, hhi,
                            alive, dq, flags, s_cnt[MULTI ? pi : 0], words[7 * nb], words[8 * nb]);
          rem = region_distance(G, out, px, py, pz, ux, uy, uz);
          has = true;
          dv = cv;
        }
        // The scattered photons tally their deposit now and take their next
        // flight step in this same iteration instead of idling through it.
        if (HIST) {
          if (has) hist_add(hl, hn, (uint32_t)dv, dq, p.g.tally, p.s2h_lo, p.s2h_hi, p.g.counters + kCtrHistSplits);
        } else {
          tally_flush<WARP_AGG>(G.tally + dv, has, dq, lane);
        }
        has = false;
        dq = 0;
        dv = 0;
      }
    }
    // ---- one Woodcock flight step per live lane -------------------------------
    if (alive && !pending_c && !has) {
      // A fresh Philox block every step (words x and y; z and w serve the
      // Compton angle if the step finds one): keeping them for the next step
      // would save draws per lane but not per warp, where lanes
      // are out of phase, and costs registers.
      const uint4 rr = draw(ctr, stream, hlo, hhi, p.key);
      const uint32_t r0 = rr.x, r1 = rr.y;
      const float imaj = f.inv_mubar;
      float s = -__logf(u01(r0)) * imaj;   // cm
      const bool cross = s >= rem;         // flight cut at the region boundary
      if (cross) s = rem;
      rem -= s;
      px = fmaf(s * G.inv_dx, ux, px);
      py = fmaf(s * G.inv_dy, uy, py);
      pz = fmaf(s * G.inv_dz, uz, pz);
      ++n_steps;
      ++steps;
      // floor once: the same integers test the grid bounds (negative or past
      // the end, as unsigned) and index the voxel (positions are finite)
      const int ix = __float2int_rd(px), iy = __float2int_rd(py), iz = __float2int_rd(pz);
      if ((unsigned)ix >= (unsigned)G.nx || (unsigned)iy >= (unsigned)G.ny || (unsigned)iz >= (unsigned)G.nz) {
        escaped += (ull)qe;
        ++n_esc;
        alive = false;
      } else if (cross) {
        out = !out;
        rem = out ? kInf : region_distance(G, false, px, py, pz, ux, uy, uz);
        f.inv_mubar = inv_majorant_at(e, out ? s_minv_out : s_minv, p.ln_e_lo, p.inv_dln_e);
      } else {
        const int v = (iz * G.ny + iy) * G.nx + ix;
        const uint32_t wv = __ldg(G.vox + v);
        const MaterialCoef c = s_mat[wv & 7u];
        // real event with probability mu(voxel)/mubar; the same uniform picks the type
        const float scale = __uint_as_float(wv & ~7u) * imaj;
        const float ic = c.za * f.s_c;
        const float icp = fmaf(c.zp, f.s_pe, ic);
        const float t = u01(r1);
        if (t < scale * ic) {
          ++n_compton;
          if (REGROUP) {
            pending_c = true;
            cv = v;
            // the step's two unused words wait in the stash for the Compton pass
            uint32_t* words = reinterpret_cast<uint32_t*>(site);
            words[7 * nb] = rr.z;
            words[8 * nb] = rr.w;
          } else {
            compton<RAYLEIGH>(p, s_kn, out ? s_minv_out : s_minv, e, qe, f, ux, uy, uz, ctr, stream, hlo,
                              hhi, alive, dq, flags, s_cnt[MULTI ? pi : 0], rr.z, rr.w);
            rem = region_distance(G, out, px, py, pz, ux, uy, uz);
            has = true;
            dv = v;
          }
        } else if (t < scale * icp) {
          atomicAdd(&s_cnt[MULTI ? pi : 0][kCtrPhoto], 1ull);
          has = true;
          dv = v;
          dq = (uint32_t)qe;
          alive = false;
        } else if (RAYLEIGH && t < scale * fmaf(c.zr, f.s_r, icp)) {
          atomicAdd(&s_cnt[MULTI ? pi : 0][kCtrRayleigh], 1ull);
          // Thomson angular shape (1 + cos^2)/2 by rejection; one block per trial.
          for (int trial = 0;; ++trial) {
            const uint4 r = draw(ctr, stream, hlo, hhi, p.key);
            const float cth = fmaf(2.0f, u01(r.x), -1.0f);
            const bool acc = 2.0f * u01(r.y) <= fmaf(cth, cth, 1.0f);
            if (acc || trial + 1 >= kKahnTrialLimit) {
              if (!acc) flags |= NM_DEV_RAYLEIGH_LIMIT;
              rotate(ux, uy, uz, cth, fmaf(kTwoPi, u01(r.z), -3.14159265f));
              rem = region_distance(G, out, px, py, pz, ux, uy, uz);
              break;
            }
          }
        }
      }
      if (alive && steps >= p.max_steps) {
        atomicAdd(&s_cnt[MULTI ? pi : 0][kCtrKilledUnits], (ull)qe);
        flags |= NM_DEV_STEP_LIMIT;
        alive = false;
        pending_c = false;
      }
    }
    if (HIST) {
      if (has) hist_add(hl, hn, (uint32_t)dv, dq, p.g.tally, p.s2h_lo, p.s2h_hi, p.g.counters + kCtrHistSplits);
    } else {
      tally_flush<WARP_AGG>(G.tally + dv, has, dq, lane);
    }
  }
  if (HIST && hn) hist_flush(hl, hn, p.g.tally, p.s2h_lo, p.s2h_hi);

  // ---- counters ---------------------------------------------------------------
  if (MULTI) {
    atomicAdd(&s_cnt[cpi][kCtrSteps], (ull)n_steps);
    atomicAdd(&s_cnt[cpi][kCtrCompton], (ull)n_compton);
    atomicAdd(&s_cnt[cpi][kCtrEscapes], (ull)n_esc);
    atomicAdd(&s_cnt[cpi][kCtrEscapedUnits], escaped);
  } else {
    // warp sums, one atomic per warp per counter
    ull sm = warp_sum((ull)n_steps);
    if (lane == 0 && sm) atomicAdd(p.g.counters + kCtrSteps, sm);
    sm = warp_sum((ull)n_compton);
    if (lane == 0 && sm) atomicAdd(p.g.counters + kCtrCompton, sm);
    sm = warp_sum((ull)n_esc);
    if (lane == 0 && sm) atomicAdd(p.g.counters + kCtrEscapes, sm);
    sm = warp_sum(escaped);
    if (lane == 0 && sm) atomicAdd(p.g.counters + kCtrEscapedUnits, sm);
  }
  const unsigned fl = __reduce_or_sync(kFull, flags);
  if (lane == 0 && fl) atomicOr(p.status, fl);
  __syncthreads();
  for (int i = threadIdx.x; i < n_pat * 10; i += blockDim.x) {
    const int q = i / 10, k = i % 10;   // k is the CounterSlot, 8 the positron and 9 the gamma units
    if (s_cnt[q][k])
      atomicAdd((MULTI ? s_geom[q].counters : p.g.counters) +
                    (k < 8 ? k : k == 8 ? (int)kCtrPositronUnits : (int)kCtrGammaUnits),
                s_cnt[q][k]);
  }
}

// Scattering cosines at energy e as the transport's table sampler draws them
// (counters 0..n-1 of stream 7, key k0 k1).
__global__ void check_kn_table_kernel(const TransportParams p, float e, int64_t n, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t ctr = 0;
  const uint4 r = draw(ctr, 7u, (uint32_t)i, (uint32_t)(i >> 32), p.key);
  out[i] = 1.0f - kn_table_x(p, e, r.x);
}

// Positron energies of histories 0..n-1 as the transport draws them.
__global__ void check_beta_kernel(const float* tab, int64_t n, uint32_t k0, uint32_t k1, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t ctr = 0;
  const uint4 r = draw(ctr, kStreamPositron, (uint32_t)i, (uint32_t)(i >> 32), philox_key(k0, k1));
  out[i] = beta_energy(tab, r.x);
}

__global__ void check_philox_kernel(const uint4* ctr, const uint2* key, int64_t n, uint4* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // the transport's own path: round keys from philox_key, then the rounds
  if (i < n) out[i] = philox4x32_10(ctr[i], philox_key(key[i].x, key[i].y));
}

__global__ void check_kahn_kernel(float e, int64_t n, uint32_t k0, uint32_t k1, float* out,
                                  uint32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t ctr = 0, rphi, flags = 0;
  const float x = kahn_x(e * kInvElectronMassMeV, ctr, 7u, (uint32_t)i, (uint32_t)(i >> 32), philox_key(k0, k1),
                         rphi, flags);
  out[i] = 1.0f - x;
  if (flags) atomicOr(status, flags);
}

__global__ void check_source_kernel(const TransportParams p, uint64_t first, int64_t n,
                                    int32_t* voxel, float* pos, float* dir) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t h = first + (uint64_t)i;
  const Site s = sample_site(p.g, p.key, (uint32_t)h, (uint32_t)(h >> 32));
  voxel[i] = s.v;
  pos[3 * i + 0] = s.x / p.g.inv_dx;
  pos[3 * i + 1] = s.y / p.g.inv_dy;
  pos[3 * i + 2] = s.z / p.g.inv_dz;
  dir[3 * i + 0] = s.u;
  dir[3 * i + 1] = s.v_;
  dir[3 * i + 2] = s.w;
}

// Dynamic shared memory: the site stash, the history lists when kept, and
// (nuclide variant) the origin of the gamma lines.
size_t transport_smem(int block, bool history, bool beta = false, bool siteq = false) {
  return (((size_t)9 + (history ? 2 * kHistVoxels : 0) + (beta ? 3 : 0)) * block +
          (siteq ? (size_t)(block / 32) * kQueueCap * kQueueWords : 0)) * sizeof(float);
}

template <bool A, bool R, bool G, bool M, bool H, bool B = false>
void* kernel_ptr() {
  return (void*)transport_kernel<A, R, G, M, H, B>;
}

template <bool M>
void* pick_m(bool a, bool r, bool g) {
  if (a) {
    if (r) return g ? kernel_ptr<true, true, true, M, false>() : kernel_ptr<true, true, false, M, false>();
    return g ? kernel_ptr<true, false, true, M, false>() : kernel_ptr<true, false, false, M, false>();
  }
  if (r) return g ? kernel_ptr<false, true, true, M, false>() : kernel_ptr<false, true, false, M, false>();
  return g ? kernel_ptr<false, false, true, M, false>() : kernel_ptr<false, false, false, M, false>();
}

template <bool H>
void* pick_beta(bool r, bool g) {
  if (r) return g ? kernel_ptr<false, true, true, false, H, true>() : kernel_ptr<false, true, false, false, H, true>();
  return g ? kernel_ptr<false, false, true, false, H, true>() : kernel_ptr<false, false, false, false, H, true>();
}

// History statistics and the beta+ spectrum exist only without warp
// aggregation and for one patient.
void* pick(bool a, bool r, bool g, bool m, bool h, bool beta) {
  if (beta) {
    if (a || m) return nullptr;
    return h ? pick_beta<true>(r, g) : pick_beta<false>(r, g);
  }
  if (h) {
    if (a || m) return nullptr;
    if (r) return g ? kernel_ptr<false, true, true, false, true>() : kernel_ptr<false, true, false, false, true>();
    return g ? kernel_ptr<false, false, true, false, true>() : kernel_ptr<false, false, false, false, true>();
  }
  return m ? pick_m<true>(a, r, g) : pick_m<false>(a, r, g);
}

}  // namespace

bool nuclide_launch(const TransportParams& p) {
  return p.g.beta_tab != nullptr || p.n_gamma > 0 || (p.g.source_mode == NM_SOURCE_DECAY && !p.annihilate);
}

cudaError_t launch_transport(const TransportParams& p, int grid, int block, bool warp_agg,
                             bool rayleigh, bool regroup, cudaStream_t s, bool multi, bool history) {
  const bool beta = !multi && nuclide_launch(p);
  void* fn = pick(warp_agg, rayleigh, regroup, multi, history, beta);
  if (!fn) return cudaErrorInvalidValue;
  void* args[] = {(void*)&p};
  // the history lists and the site queues take the static + dynamic total
  // past the 48 KB default
  const size_t smem = transport_smem(block, history, beta, regroup && !multi && !history && !beta);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, s);
  if (e != cudaSuccess) cudaGetLastError();  // a refused launch must not linger as the last error
  return e;
}

int transport_max_blocks_per_sm(int block, bool warp_agg, bool rayleigh, bool regroup, bool multi, bool history,
                                bool beta) {
  int n = 0;
  void* fn = pick(warp_agg, rayleigh, regroup, multi, history, beta);
  const size_t smem = transport_smem(block, history, beta, regroup && !multi && !history && !beta);
  if (!fn || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_check_kn_table(const TransportParams& p, float e, int64_t n, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_kn_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, e, n, out);
  return cudaGetLastError();
}

cudaError_t launch_check_beta(const float* tab, int64_t n, uint32_t k0, uint32_t k1, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_beta_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tab, n, k0, k1, out);
  return cudaGetLastError();
}

cudaError_t launch_check_philox(const uint4* ctr, const uint2* key, int64_t n, uint4* out,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctr, key, n, out);
  return cudaGetLastError();
}

cudaError_t launch_check_kahn(float e, int64_t n, uint32_t k0, uint32_t k1, float* out,
                              uint32_t* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_kahn_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(e, n, k0, k1, out, status);
  return cudaGetLastError();
}

cudaError_t launch_check_source(const TransportParams& p, uint64_t first, int64_t n, int32_t* voxel,
                                float* pos, float* dir, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_source_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, first, n, voxel, pos, dir);
  return cudaGetLastError();
}

}  // namespace nm
