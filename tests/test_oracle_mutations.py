"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy
of the oracle's C source (on the CPU, in a temporary directory), rebuilds it there and
runs the pin suites against it; they must fail.  A representative ten of the mistakes
the pins were checked against (signs, weights, windows, caps, the tie rule, a dropped
margin, the rotation order)."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MISTAKES = {
    "tie_to_larger_address": ("(m == r->m_best && H[j].addr < H[best].addr)",
                              "(m == r->m_best && H[j].addr > H[best].addr)"),
    "vertex_z_unweighted": ("wz += zi[i] / vi[i]; wzs += 1.0 / vi[i];", "wz += zi[i]; wzs += 1.0;"),
    "vertex_chi2_without_z": ("chi2 += (dx * dx + dy * dy + dz * dz) / vi[i];",
                              "chi2 += (dx * dx + dy * dy) / vi[i];"),
    "target_margin_dropped": ("double lim = c->target_r + c->isect_margin;", "double lim = c->target_r;"),
    "theta_kink_sign": ("f->beta = f->dtheta[1] - f->dtheta[0];", "f->beta = f->dtheta[1] + f->dtheta[0];"),
    "kappa_bar_unweighted": ("double kb = (t1->kappa * w1 + t2->kappa * w2) / (w1 + w2);",
                             "double kb = 0.5 * (t1->kappa + t2->kappa);"),
    "rtc_without_half": ("f->rtc = d01 * d12 * d20 / (2.0 * cross);", "f->rtc = d01 * d12 * d20 / cross;"),
    "phi01_cut_sine": ("return v[1] >= cos(c->phi01_max);", "return v[1] >= sin(c->phi01_max);"),
    "triplet_cap_off_by_one": ("if (ntrip > c->max_triplets) {", "if (ntrip >= c->max_triplets) {"),
    "rotation_transposed": (
        "x[i] = R[3 * i] * xn[0] + R[3 * i + 1] * xn[1] + R[3 * i + 2] * xn[2] + p6[i];",
        "x[i] = R[i] * xn[0] + R[3 + i] * xn[1] + R[6 + i] * xn[2] + p6[i];"),
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_pins_catch_a_planted_mistake(name, tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc is missing")
    old, new = MISTAKES[name]
    ignore = shutil.ignore_patterns("*.so", "*.o", "__pycache__", "csrc", ".pytest_cache")
    for sub in ("oracle", "tests", "paper_2206_11535_gb300"):
        shutil.copytree(os.path.join(ROOT, sub), tmp_path / sub, ignore=ignore)
    src = tmp_path / "oracle" / "m3e_oracle.c"
    text = src.read_text()
    assert text.count(old) == 1, name
    src.write_text(text.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "tests/test_oracle_fit_grad.py",
                        "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, (name, r.stdout[-2000:], r.stderr[-2000:])
