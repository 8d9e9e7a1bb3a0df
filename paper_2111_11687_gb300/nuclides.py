"""Decay data of the radionuclides the engine is set up for, as nm_options
keyword arguments of ``nmdose.Dose`` / ``nmdose.options``.

The paper simulates 18F (§2.1: every decay gives a positron whose two 0.511
MeV annihilation photons are transported) and names 177Lu and 131I as the
next radionuclides (§4).  Values are the published ones (NNDC NuDat, ICRP
Publication 107): beta branches as (endpoint MeV, fraction of decays), the
daughter's atomic number for the Fermi function, and the main gamma lines as
(MeV, photons per decay).  X-rays and conversion electrons are left out.

    from paper_2111_11687_gb300 import nmdose, nuclides
    d = nmdose.Dose(density, material, spacing, materials, activity=act, **nuclides.LU177)
"""

# 18F -> 18O: positron emitter (endpoint 0.6335 MeV, 96.9 % beta+); the
# default decay of the engine deposits the mean positron energy locally.
F18 = dict(photon_mev=0.511, positron_mev=0.25)

# 18F with the positron's energy drawn from its spectrum and its range tracked.
F18_TRACKED = dict(photon_mev=0.511, beta_max_mev=0.6335, beta_z=8)

# 177Lu -> 177Hf: beta- (mean 133.6 keV per decay), gamma 208.4 and 113.0 keV.
LU177 = dict(no_annihilation=1, beta_electron=1, beta_z=72, positron_mev=0.0,
             beta_branches=[(0.4983, 0.794), (0.3849, 0.091), (0.1765, 0.116)],
             gamma_lines=[(0.2084, 0.104), (0.1130, 0.062)])

# 131I -> 131Xe: beta- (mean 181.9 keV per decay), gamma 364.5 keV and others.
I131 = dict(no_annihilation=1, beta_electron=1, beta_z=54, positron_mev=0.0,
            beta_branches=[(0.6063, 0.896), (0.3338, 0.0723), (0.2479, 0.0208), (0.8069, 0.0039)],
            gamma_lines=[(0.3645, 0.815), (0.6370, 0.0716), (0.2843, 0.0612), (0.0802, 0.0262),
                         (0.7229, 0.0177)])

# Physical half-lives in hours (for nm_time_integrated_activity).
HALF_LIFE_H = {"18F": 109.77 / 60.0, "177Lu": 6.647 * 24.0, "131I": 8.0252 * 24.0}
