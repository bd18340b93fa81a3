"""The oracle's pins must be sensitive: each plausible slip below, planted in
a temporary copy of the oracle's C source (on the CPU, never in the
repository), must make at least one pin in ``test_oracle_pins`` fail."""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "gjp_oracle.c")

MUTANTS = {
    "wrong tap pattern (Eq. 12)": ("{&pfl[0], &pcl[1], &pcl[2]},", "{&pfl[0], &pfl[1], &pcl[2]},"),
    "no step factor": ("const double step = sqrt(hr2);", "const double step = 1.0;"),
    "sign of the sampling offset (Eq. 5)": ("const double o = -s[m];", "const double o = s[m];"),
    "complementary weight (Eq. 11)": ("wcl[k] = 1.0 - wfl[k];", "wcl[k] = wfl[k];"),
    "argmin instead of argmax (Eq. 3)": ("if (fabs(r[k]) > fabs(r[m])) m = k;",
                                         "if (fabs(r[k]) < fabs(r[m])) m = k;"),
    "transposed memory layout": ("const int64_t idx = (i * V->n[1] + j) * V->n[2] + k;",
                                 "const int64_t idx = (k * V->n[1] + j) * V->n[0] + i;"),
    "w_lin weight on the wrong neighbour (Eq. 13)": ("return 1.0 - d;\n}", "return d;\n}"),
    "first plane dropped": ("for (int64_t i = 0; i < imax; ++i) {", "for (int64_t i = 1; i < imax; ++i) {"),
    "zero border read as clamp": ("if (v < 0.0 || v > (double)(V->n[k] - 1)) inside = 0;",
                                  "if (0) inside = 0;"),
}


def _checks():
    return [
        lambda: [pins.test_axis_aligned_ray_is_column_sum(a) for a in (0, 1, 2)],
        pins.test_constant_volume_gives_exact_chord_length,
        pins.test_affine_field_integral_closed_form,
        lambda: pins.test_branchless_equals_textbook_joseph(0, True),
        pins.test_increment_bounds,
        pins.test_zero_border_partial_contribution,
        pins.test_ray_missing_the_volume_is_zero,
    ]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name!r} not unique"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    so = tmp_path / "mutant.so"
    # "zero border read as clamp" would index out of range: clamp the index
    # in the mutant so it stays a memory-safe wrong answer
    if name == "zero border read as clamp":
        src.write_text(src.read_text().replace(
            "idx[k] = inside ? (int64_t)v : 0;",
            "idx[k] = v < 0 ? 0 : (v > (double)(V->n[k] - 1) ? V->n[k] - 1 : (int64_t)v);"))
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-std=c11", "-shared", "-fPIC",
                           "-o", str(so), str(src), "-lm"])
    saved = oracle._load()
    oracle._lib = oracle._open(str(so))
    caught = []
    try:
        for check in _checks():
            try:
                check()
            except (AssertionError, ValueError, IndexError):
                caught.append(check)
    finally:
        oracle._lib = saved
    assert caught, f"no pin caught the planted mistake: {name}"
