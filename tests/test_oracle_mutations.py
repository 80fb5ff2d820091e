"""The oracle's pins have teeth: each plausible mistake below, planted in a
scratch copy of the oracle's C source on the CPU, makes at least one of the
pin tests fail.  The real oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name: (original text, planted mistake, pin test files expected to catch it)
MUTATIONS = {
    "threshold uses dE/2": (
        "const double p = exp(-beta * dE);", "const double p = exp(-beta * dE * 0.5);",
        ["test_oracle_acceptance.py"]),
    "wrong vertical neighbour": (
        "s[up1(y, L) * L + x] + s[dn1(y, L) * L + x];",
        "s[up1(y, L) * L + x] + s[up1(y, L) * L + x];",
        ["test_oracle_acceptance.py", "test_oracle_equilibrium.py"]),
    "Blume-Capel proposal order swapped": (
        "return b ? +1 : -1;", "return b ? -1 : +1;", ["test_oracle_acceptance.py"]),
    "comparison reversed": (
        "accept = (uint64_t)u < threshold_bits(beta, dE, 32);",
        "accept = (uint64_t)u >= threshold_bits(beta, dE, 32);",
        ["test_oracle_acceptance.py"]),
    "crystal-field sign": (
        "+ delta * (double)(s2 * s2 - s * s)", "- delta * (double)(s2 * s2 - s * s)",
        ["test_oracle_acceptance.py", "test_oracle_equilibrium.py"]),
    "bond sum misses vertical bonds": (
        "(s[y * L + up1(x, L)] + s[up1(y, L) * L + x])",
        "(s[y * L + up1(x, L)] + s[y * L + up1(x, L)])",
        ["test_oracle_observables.py"]),
    "Philox key increment": (
        "k[1] += 0xBB67AE85u;", "k[1] += 0xBB67AE84u;", ["test_oracle_philox.py"]),
    "correlation partner off by one": (
        "ax += v * s[y * L + (x + r[k]) % L];", "ax += v * s[y * L + (x + r[k] + 1) % L];",
        ["test_oracle_correlation.py"]),
    "Swendsen-Wang bonds anti-aligned pairs": (
        "if (s[jx] == s[i] && (uint64_t)full_index_word(seed, (uint64_t)i, (uint32_t)k, 4) < thr)",
        "if (s[jx] != 0 && (uint64_t)full_index_word(seed, (uint64_t)i, (uint32_t)k, 4) < thr)",
        ["test_oracle_swendsen_wang.py"]),
    "Swendsen-Wang bond probability 1 - exp(-beta)": (
        "ldexp(-expm1(-2.0 * beta), 32)", "ldexp(-expm1(-1.0 * beta), 32)",
        ["test_oracle_swendsen_wang.py"]),
    "Swendsen-Wang coin per site instead of per cluster": (
        "full_index_word(seed, (uint64_t)parent[i], (uint32_t)k, 6)",
        "full_index_word(seed, (uint64_t)i, (uint32_t)k, 6)",
        ["test_oracle_swendsen_wang.py"]),
    "hot-start bias": (
        "s[idx] = (int8_t)(u >= 0x80000000u ? 1 : -1);",
        "s[idx] = (int8_t)(u >= 0x7F000000u ? 1 : -1);",
        ["test_oracle_acceptance.py"]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    original, planted, files = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "isg_oracle.c")).read()
    assert src.count(original) == 1, "mutation anchor no longer in the oracle source"
    work = tmp_path / "copy"
    shutil.copytree(os.path.join(ROOT, "oracle"), work / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), work / "tests",
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py"))
    (work / "oracle" / "isg_oracle.c").write_text(src.replace(original, planted))
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           *[os.path.join("tests", f) for f in files]]
    r = subprocess.run(cmd, cwd=work, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"planted mistake '{name}' was not caught:\n{r.stdout[-2000:]}"
    assert " failed" in r.stdout
