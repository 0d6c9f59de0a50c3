"""Closed-form relations of the paper used as physics pins (TEST INFRASTRUCTURE).

- Relativistic Harris sheet (App. C, Eq. velocity_Harris and Eq. pressure_ad)
  for a pair plasma with equal temperatures (chi = 1): Theta = (omega_ce /
  omega'_pe)^2 / 4 and Gamma U / c = 2 Theta (d'_e / L)(omega'_pe / omega_ce);
  lab-frame plasma frequency omega_pe = sqrt(Gamma) omega'_pe (Sect. 3.4).
- Cold filamentation growth time for k_perp -> infinity (Sect. 3.2.1):
  tau = (1/2 pi) sqrt(Gamma0 / 2) / beta0 T_pe for pair beams.  The same cold
  two-fluid limit, delta^2 = sum_s omega_ps^2 beta_s^2 / gamma_s over the beam
  populations, gives tau = (1/2 pi) sqrt(Gamma0) / beta0 T_pe for two electron
  beams of half density each on a positron background at rest.
- Cold filamentation at a finite wavenumber (Sect. 3.2.1's cold setting):
  for cold populations s streaming along z with beta_s, gamma_s and plasma
  frequencies omega_ps, a perturbation E_z, B_y ~ exp(i k x + delta t) with k
  across the flow obeys (cold relativistic two-fluid equations and Maxwell's
  equations, lengths in c / omega_pe, rates in omega_pe)
      delta^4 + (k^2 + A) delta^2 - k^2 C = 0,
      A = sum_s omega_ps^2 / gamma_s^3,   C = sum_s omega_ps^2 beta_s^2 / gamma_s.
  Its positive root grows with k towards sqrt(C), the k -> infinity rate that
  the paper's tau formula states.
- Unmagnetized thermal modes (Sect. 3.1.1): the transverse electromagnetic
  wave omega^2 = omega_P^2 + k^2 c^2 and the Langmuir wave
  omega^2 = omega_P^2 (1 + 3 k^2 lambda_D^2), lambda_D = v_th / omega_pe, with
  omega_P = omega_pe (1 + m_e/m_i)^1/2.
- k = 0 pulsations of a cold magnetized electron-ion plasma (Sect. 3.1.2):
  omega_P along B0, and the cut-offs omega_L, omega_R across it.  With
  infinitely heavy ions omega_{L,R} = [(omega_ce^2 + 4 omega_pe^2)^1/2 -/+
  omega_ce] / 2 (the paper's formulas).  With mobile ions they are the
  positive roots of the cold-plasma conditions L(omega) = 0 and R(omega) = 0,
  R = 1 - sum_s omega_ps^2 / (omega (omega + Omega_s)), L(omega) = R(-omega),
  Omega_s = q_s B / m_s signed, omega_pi^2 = omega_pe^2 m_e / m_i.
"""
import numpy as np


def harris_from_theta_GU(theta, GU):
    """(omega_ce/omega_pe, L/d_e) in lab-frame units from Theta and Gamma_e U_e / c."""
    G = np.sqrt(1.0 + GU * GU)
    wce_over_wpe_prime = 2.0 * np.sqrt(theta)        # pressure balance, chi = 1
    L_over_dprime = 2.0 * theta / (GU * wce_over_wpe_prime)
    return wce_over_wpe_prime / np.sqrt(G), L_over_dprime * np.sqrt(G)


def tau_filamentation_pair(beta0):
    G0 = 1.0 / np.sqrt(1.0 - beta0 * beta0)
    return np.sqrt(G0 / 2.0) / beta0 / (2.0 * np.pi)


def tau_filamentation_electron_beams(beta0):
    G0 = 1.0 / np.sqrt(1.0 - beta0 * beta0)
    return np.sqrt(G0) / beta0 / (2.0 * np.pi)


def filamentation_rate_cold(kc, populations):
    """delta / omega_pe of the purely growing filamentation mode at kc = k c /
    omega_pe across the flow.  populations: iterable of (wp2, beta, gamma) with
    wp2 = omega_ps^2 / omega_pe^2 (density and mass of population s relative to
    the electrons that define omega_pe).  The positive root in delta^2 of
    delta^4 + (k^2 + A) delta^2 - k^2 C = 0 (module docstring)."""
    A = sum(w / g ** 3 for w, b, g in populations)
    C = sum(w * b * b / g for w, b, g in populations)
    k2 = kc * kc
    p = k2 + A
    # the positive root (sqrt(p^2 + 4 k^2 C) - p) / 2, written without cancellation
    d2 = 2.0 * k2 * C / (np.sqrt(p * p + 4.0 * k2 * C) + p)
    return np.sqrt(d2)


def cold_plasma_frequency(mass_ratio):
    """omega_P / omega_pe of an electron-ion plasma with m_i / m_e = mass_ratio."""
    return np.sqrt(1.0 + 1.0 / mass_ratio)


def cold_cutoffs_heavy_ions(wce):
    """(omega_L, omega_R) / omega_pe for infinitely heavy ions; wce = omega_ce / omega_pe."""
    s = np.sqrt(wce * wce + 4.0)
    return 0.5 * (s - wce), 0.5 * (s + wce)


def cold_cutoffs_two_species(wce, mass_ratio):
    """(omega_L, omega_R) / omega_pe with ions of mass mass_ratio * m_e: the
    positive roots of R(omega) = 0, multiplied out to the cubic
    omega (omega - wce)(omega + wci) - (omega + wci) - (omega - wce) / mass_ratio = 0,
    wci = wce / mass_ratio.  Its roots are omega_R, 0 and -omega_L (L(omega) = R(-omega))."""
    wci = wce / mass_ratio
    cubic = (np.poly1d([1.0, -wce, 0.0]) * np.poly1d([1.0, wci]) - np.poly1d([1.0, wci])
             - np.poly1d([1.0, -wce]) / mass_ratio)
    roots = np.sort(cubic.roots.real)
    return -roots[0], roots[-1]


def transverse_wave(kc, mass_ratio):
    """omega / omega_pe of the transverse wave at wavenumber kc = k c / omega_pe."""
    return np.sqrt(1.0 + 1.0 / mass_ratio + kc * kc)


def langmuir_wave(k_lambda, mass_ratio):
    """omega / omega_pe of the thermal Langmuir wave at k lambda_D (lambda_D = v_th/omega_pe)."""
    return np.sqrt((1.0 + 1.0 / mass_ratio) * (1.0 + 3.0 * k_lambda * k_lambda))
