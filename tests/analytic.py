"""Closed-form Debye-Hueckel / Stokes results of the paper, used as pins.

Lattice units (k_B T = e = 1); eps = 1/(4 pi l_B) stands for eps0*epsr and
kappa = 1/lambda_D.
"""
import math

import numpy as np
from scipy.special import iv, kv


def eps_of(bjerrum):
    return 1.0 / (4.0 * math.pi * bjerrum)


def dh_plate_potential(z, L, kappa, psi1, psi2):
    """Eq. DHslitpotential; z measured from the mid-plane, electrodes at -L/2
    (psi1) and +L/2 (psi2)."""
    return 0.5 * (psi1 + psi2) + 0.5 * (psi2 - psi1) * np.sinh(kappa * z) / np.sinh(kappa * L / 2.0)


def dh_plate_charge_per_area(eps, kappa, L, dpsi):
    """Surface charge of the positive plate from the field of Eq.
    DHslitpotential at z = L/2: eps * kappa * (dpsi/2) * coth(kappa L/2).
    For lambda_D << L it tends to C_DH * dpsi with C_DH = eps/(2 lambda_D)
    (Eq. SLITcapaDH)."""
    return eps * kappa * 0.5 * dpsi / math.tanh(kappa * L / 2.0)


def dielectric_plate_charge_per_area(eps, L, dpsi):
    """C_0 = eps/L for the neutral liquid (Sec. "Charge and capacitance")."""
    return eps * dpsi / L


def dh_plate_eof(z, L, kappa, eps, eta, E, dpsi):
    """Eq. DHslitEOF: steady electro-osmotic velocity along the field."""
    return eps * E * dpsi / eta * 0.5 * (np.sinh(kappa * z) / np.sinh(kappa * L / 2.0) - 2.0 * z / L)


def coax_log_potential(r, R1, R2, psi1, psi2):
    """Eq. PSIcoxialNosalt (neutral liquid)."""
    return psi1 + (psi2 - psi1) * np.log(r / R1) / math.log(R2 / R1)


def coax_f(r, R1, R2, kappa):
    """Eq. PSIcoxialDH2."""
    k = kappa
    a = R2 * kv(1, k * R2) - R1 * kv(1, k * R1)
    b = R2 * iv(1, k * R2) - R1 * iv(1, k * R1)
    num = a * (iv(0, k * r) - iv(0, k * R1)) + b * (kv(0, k * r) - kv(0, k * R1))
    den = a * (iv(0, k * R2) - iv(0, k * R1)) + b * (kv(0, k * R2) - kv(0, k * R1))
    return num / den


def coax_dh_potential(r, R1, R2, kappa, psi1, psi2):
    """Eq. PSIcoxialDH."""
    return psi1 + (psi2 - psi1) * coax_f(r, R1, R2, kappa)


def coax_c0_per_length(eps, R1, R2):
    """C_0^cyl = 2 pi eps / ln(R2/R1)."""
    return 2.0 * math.pi * eps / math.log(R2 / R1)


def coax_cdh_per_length(eps, R1, R2, kappa):
    """Eq. CYLcapaDH: 2 pi eps R1 f'(R1)."""
    k = kappa
    a = R2 * kv(1, k * R2) - R1 * kv(1, k * R1)
    b = R2 * iv(1, k * R2) - R1 * iv(1, k * R1)
    den = a * (iv(0, k * R2) - iv(0, k * R1)) + b * (kv(0, k * R2) - kv(0, k * R1))
    # d/dr I0(k r) = k I1(k r); d/dr K0(k r) = -k K1(k r)
    fprime = (a * k * iv(1, k * R1) - b * k * kv(1, k * R1)) / den
    return 2.0 * math.pi * eps * R1 * fprime


def coax_dh_eof(r, R1, R2, kappa, eps, eta, E, dpsi):
    """Eq. DHcoaxialEOF."""
    return eps * E * dpsi / eta * (coax_f(r, R1, R2, kappa) - np.log(r / R1) / math.log(R2 / R1))
