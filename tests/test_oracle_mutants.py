"""Mutation tests: each build of the oracle with one planted mistake must fail
at least one pin. This shows that the pins constrain every step of the oracle
(quantizer, random numbers, gradient, step size, threshold, backtracking).
Mistakes are planted only in the CPU oracle, through its QO_MUTANT switch."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# mutant id -> (what it breaks, pins expected to catch it)
MUTANTS = {
    1: ("rounding-up test reversed (u > f)", "test_round_up_probability or test_unbiased"),
    2: ("grid half-width L/2 instead of (L-1)/2", "test_codes_on_grid"),
    3: ("gradient formed with the second quantization", "test_gradient_uses_first_matrix"),
    4: ("step-size numerator not squared", "test_sparsity_and_step_size_bounds"),
    5: ("H_s keeps the smallest entries", "test_top_s_matches or test_exact_recovery"),
    6: ("backtracking condition reversed", "test_backtracking_condition"),
    7: ("Philox key schedule dropped", "test_philox_matches_triton or test_philox_avalanche"),
    8: ("residual sign flipped", "test_exact_recovery or test_brute_force_noiseless"),
    9: ("dequantised level off by one", "test_codes_on_grid or test_unbiased"),
    10: ("cross step size formed with the second quantization twice", "test_cross_is_unbiased"),
    11: ("residual tolerance test reversed", "test_tol_stops_exact_recovery_early"),
    12: ("e4m3 residual with its third term dropped", "test_e4m3_terms_error_bound"),
    13: ("e4m3 residual scaled one binade too high (saturates)", "test_e4m3_terms_error_bound"),
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_mutant(mutant, tmp_path):
    if mutant == 7:
        pytest.importorskip("triton")
    lib = oracle.build(force=True, mutant=mutant, out=str(tmp_path / f"libqiht_oracle_m{mutant}.so"))
    what, sel = MUTANTS[mutant]
    env = {**os.environ, "QIHT_ORACLE_LIB": lib}
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_oracle_rng.py"),
           os.path.join(ROOT, "tests", "test_oracle_quantizer.py"),
           os.path.join(ROOT, "tests", "test_oracle_niht.py"),
           os.path.join(ROOT, "tests", "test_oracle_step_modes.py"),
           os.path.join(ROOT, "tests", "test_oracle_e4m3.py"), "-k", sel]
    out = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert "passed" in out.stdout or "failed" in out.stdout, out.stdout[-500:] + out.stderr[-500:]
    assert out.returncode != 0, f"mutant {mutant} ({what}) passed every selected pin:\n{out.stdout[-800:]}"


def test_unmutated_oracle_passes_the_same_selection(tmp_path):
    lib = oracle.build(force=True, mutant=0, out=str(tmp_path / "libqiht_oracle_m0.so"))
    sel = " or ".join(s for _, s in MUTANTS.values())
    env = {**os.environ, "QIHT_ORACLE_LIB": lib}
    cmd = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_oracle_rng.py"),
           os.path.join(ROOT, "tests", "test_oracle_quantizer.py"),
           os.path.join(ROOT, "tests", "test_oracle_niht.py"),
           os.path.join(ROOT, "tests", "test_oracle_step_modes.py"),
           os.path.join(ROOT, "tests", "test_oracle_e4m3.py"), "-k", sel]
    out = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-1500:]
