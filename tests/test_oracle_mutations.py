"""Each plausible slip planted in a copy of the oracle must fail the pins.

The mutants are text edits of a temporary copy of ``oracle/spgpe_oracle.cpp``
(on the CPU only); for each, the fast pin suite runs in a subprocess against
the mutated copy and must report a failure.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "soc_sign": [("const double tu = k2 - m->kL * kx, td = k2 + m->kL * kx;",
                  "const double tu = k2 + m->kL * kx, td = k2 - m->kL * kx;")],
    "raman_sign": [("const cd mis(0.0, -s);", "const cd mis(0.0, s);")],
    "raman_half_angle": [("const double a = 0.5 * m->Omega[i] * tau;",
                          "const double a = m->Omega[i] * tau;")],
    "g11_g22_swapped": [("const double eu = v + 0.5 * d + m->g11 * ru",
                         "const double eu = v + 0.5 * d + m->g22 * ru"),
                        ("const double ed = v - 0.5 * d + m->g22 * rd",
                         "const double ed = v - 0.5 * d + m->g11 * rd")],
    "g12_own_density": [("+ m->g12 * rd;\n    const double ed", "+ m->g12 * ru;\n    const double ed")],
    "detuning_sign": [("const double eu = v + 0.5 * d", "const double eu = v - 0.5 * d"),
                      ("const double ed = v - 0.5 * d", "const double ed = v + 0.5 * d")],
    "time_reversed": [("std::polar(1.0, -tau * eu)", "std::polar(1.0, tau * eu)"),
                      ("std::polar(1.0, -tau * ed)", "std::polar(1.0, tau * ed)"),
                      ("std::polar(1.0, -tau * tu)", "std::polar(1.0, tau * tu)"),
                      ("std::polar(1.0, -tau * td)", "std::polar(1.0, tau * td)"),
                      ("const cd mis(0.0, -s);", "const cd mis(0.0, s);")],
    "d_outer_split": [("  apply_X(m, up, dn, 0.5 * tau, imag);\n  apply_D(m, up, dn, tau, imag);\n"
                       "  apply_X(m, up, dn, 0.5 * tau, imag);",
                       "  apply_D(m, up, dn, 0.5 * tau, imag);\n  apply_X(m, up, dn, tau, imag);\n"
                       "  apply_D(m, up, dn, 0.5 * tau, imag);")],
    "lie_not_strang": [("    apply_R(m, up, dn, 0.5 * dt, imag);\n    fft2d(up",
                        "    apply_R(m, up, dn, dt, imag);\n    fft2d(up"),
                       ("    fft2d(dn, m->nx, m->ny, +1);\n    apply_R(m, up, dn, 0.5 * dt, imag);\n    if (imag)",
                        "    fft2d(dn, m->nx, m->ny, +1);\n    if (imag)")],
    "per_component_ignored": [("if (norm_mode == 1) {", "if (norm_mode == 7) {")],
    "nyquist_positive": [("const int f = (i < n / 2) ? i : i - n;", "const int f = (i <= n / 2) ? i : i - n;")],
    "kinetic_factor": [("const double k2 = 0.5 * (kx * kx + ky * ky);\n      const double tu",
                        "const double k2 = (kx * kx + ky * ky);\n      const double tu")],
    "density_after_update": [("    const double eu = v + 0.5 * d + m->g11 * ru + m->g12 * rd;\n    const double ed",
                              "    const double eu = v + 0.5 * d + m->g11 * ru + m->g12 * rd;\n"
                              "    if (imag) up[i] *= std::exp(-tau * eu);\n    const double ed")],
    "twiddle_direction": [("const double t = sign * 2.0 * kPi * m / n;", "const double t = -2.0 * kPi * m / n;")],
    "energy_raman_half": [("eram += at(m->Omega, i) * std::real(std::conj(up[i]) * dn[i]);",
                           "eram += 0.5 * at(m->Omega, i) * std::real(std::conj(up[i]) * dn[i]);")],
    "energy_g12_half": [("+ m->g12 * ru * rd;\n  }", "+ 0.5 * m->g12 * ru * rd;\n  }")],
    # Sec. 6 observables and annealing noise (pinned in test_oracle_observables.py)
    "separation_no_sqrt": [("out[0] = 1.0 - a / std::sqrt(b * c);", "out[0] = 1.0 - a / (b * c);")],
    "winding_clockwise": [("const double th = 2.0 * kPi * (double)(k % npts) / npts;",
                           "const double th = -2.0 * kPi * (double)(k % npts) / npts;")],
    "contour_90_percent": [("if (cum >= 0.99 * tot) {", "if (cum >= 0.9 * tot) {")],
    "noise_variance_doubled": [("const double r = std::sqrt(-std::log(1.0 - u1));",
                                "const double r = std::sqrt(-2.0 * std::log(1.0 - u1));")],
    "splitmix_counter_from_zero": [("unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;",
                                    "unsigned long long z = seed + c * 0x9E3779B97F4A7C15ull;")],
}
PIN_FILES = {name: "tests/test_oracle_observables.py" for name in
             ("separation_no_sqrt", "winding_clockwise", "contour_90_percent", "noise_variance_doubled",
              "splitmix_counter_from_zero")}
# the same slips against the printed gauge-potential minima alone (test_oracle_golden.py)
for _name in ("raman_half_angle", "soc_sign", "kinetic_factor"):
    MUTANTS["golden_" + _name] = MUTANTS[_name]
    PIN_FILES["golden_" + _name] = "tests/test_oracle_golden.py"


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_kill_mutant(tmp_path, name):
    src = open(os.path.join(ROOT, "oracle", "spgpe_oracle.cpp")).read()
    for a, b in MUTANTS[name]:
        assert a in src, f"mutation anchor for {name} no longer matches the oracle"
        src = src.replace(a, b)
    for d in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
    os.makedirs(tmp_path / "paper_2010_15069_gb300")
    for f in ("__init__.py", "_lib.py", "inputs.py"):
        shutil.copy(os.path.join(ROOT, "paper_2010_15069_gb300", f), tmp_path / "paper_2010_15069_gb300" / f)
    (tmp_path / "oracle" / "spgpe_oracle.cpp").write_text(src)
    r = subprocess.run([sys.executable, "-m", "pytest", PIN_FILES.get(name, "tests/test_oracle_pins.py"), "-x", "-q",
                        "-m", "not slow", "-p", "no:cacheprovider"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"mutant {name} survived:\n{r.stdout[-2000:]}"
