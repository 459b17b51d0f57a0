"""The pins catch plausible mistakes: each test compiles a copy of the oracle
with one planted error (a sign, a dropped term, a transposed index, the wrong
threshold rule), runs a pin against it on the CPU and checks that the pin
fails."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import oracle as orc_mod
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(orc_mod.__file__), "lrstv_oracle.c")
HDR = os.path.join(os.path.dirname(orc_mod.__file__), "lrstv_oracle.h")

MUTATIONS = {
    # adjoint reads the forward neighbour instead of the backward one
    "adjoint_direction": ("(i + n1 - 1) % n1", "(i + 1) % n1", "test_diff_adjoint_identity"),
    # P_z with w_n instead of w_n^2
    "pz_weight_square": ("pz[v] += w[n] * w[n] * ", "pz[v] += w[n] * ", "test_pz_closed_form"),
    # V^H without the conjugate
    "svt_missing_conj": ("* conj(V[(size_t)c + (size_t)nc * i]);", "* V[(size_t)c + (size_t)nc * i];",
                         "test_svt_matrix_vs_numpy"),
    # Gamma4 update with the wrong sign
    "gamma4_sign": ("G4[v] += mu * (E[v] - F[v]);", "G4[v] += mu * (F[v] - E[v]);",
                    "test_admm_iterations_brute_force"),
    # L-update with Gamma1 and Gamma2 swapped
    "l_update_swap": ("(G1[v] - G2[v]) / mu", "(G2[v] - G1[v]) / mu", "test_admm_iterations_brute_force"),
    # DFT with the conjugate twiddle
    "dft_sign": ("cos(ang) + (double)sign * sin(ang) * I", "cos(ang) - (double)sign * sin(ang) * I",
                 "test_dft_matches_fft"),
    # isotropic threshold: a component left out of the group norm
    "iso_norm_component": ("for (int i = 0; i < m; ++i) s += x[i] * x[i];",
                           "for (int i = 1; i < m; ++i) s += x[i] * x[i];",
                           "test_group_soft_is_the_prox_of_the_two_norm"),
    # isotropic F-update thresholding each component on its own (the anisotropic rule)
    "iso_per_component": ("orc_group_soft(x, 3, thr);",
                          "for (int c = 0; c < 3; ++c) x[c] = orc_soft(x[c], thr);",
                          "test_iso_admm_iterations_brute_force"),
    # inverse DFT without the 1/n factor
    "idft_normalisation": ("double scale = sign > 0 ? 1.0 / (double)n : 1.0;", "double scale = 1.0;",
                           "test_dft_roundtrip_parseval_symmetry"),
    # the soft threshold's second case as printed (x < d instead of x < -d)
    "soft_negative_branch": ("if (x < -d) return x + d;", "if (x < d) return x + d;",
                             "test_soft_threshold_prox"),
    # Z-solve denominator without mu on the identity term
    "zsolve_mu": ("double d = mu + mu * pz[v];", "double d = 1.0 + mu * pz[v];",
                  "test_zsolve_dense_brute_force"),
    # E-step threshold alpha instead of alpha / mu
    "e_threshold_mu": ("orc_tsvt(B, n1, n2, n3, p[ORC_P_ALPHA] / mu,", "orc_tsvt(B, n1, n2, n3, p[ORC_P_ALPHA],",
                       "test_admm_iterations_brute_force"),
    # S-update threshold lambda instead of lambda / mu
    "s_threshold_mu": ("double thr = p[ORC_P_LAMBDA] / mu;", "double thr = p[ORC_P_LAMBDA];",
                       "test_admm_iterations_brute_force"),
    # S-update with the multiplier subtracted
    "s_multiplier_sign": ("orc_soft(Y[v] - L[v] + G1[v] / mu, thr)", "orc_soft(Y[v] - L[v] - G1[v] / mu, thr)",
                          "test_admm_iterations_brute_force"),
    # Gamma3 update with the wrong sign
    "gamma3_sign": ("G3[v] += mu * (g[v] - F[v]);", "G3[v] += mu * (F[v] - g[v]);",
                    "test_admm_iterations_brute_force"),
}


def _build(tmp_path, old, new):
    src = open(SRC).read()
    assert old in src, old
    d = tmp_path / "m"
    d.mkdir()
    (d / "lrstv_oracle.c").write_text(src.replace(old, new, 1))
    shutil.copy(HDR, d / "lrstv_oracle.h")
    so = d / "lib.so"
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-std=gnu11", "-o", str(so), str(d / "lrstv_oracle.c"), "-lm"])
    return orc_mod.load_library(str(so))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, monkeypatch, name):
    old, new, pin = MUTATIONS[name]
    mutated = _build(tmp_path, old, new)
    monkeypatch.setattr(orc_mod, "_lib", mutated)
    fn = getattr(pins, pin)
    params = {
        "test_diff_adjoint_identity": {"shape": (5, 4, 3)},
        "test_svt_matrix_vs_numpy": {"m": 9, "n": 6},
        "test_iso_admm_iterations_brute_force": {"exact": False},
    }.get(pin, {})
    with pytest.raises(AssertionError):
        fn(oracle, **params)
