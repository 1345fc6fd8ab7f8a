"""The oracle's pins catch plausible mistakes: each case below plants one
mistake in a copy of oracle/leiden_oracle.c (a flipped sign, a dropped term,
a transposed operand, a wrong index, a missing guard), builds it, and runs the
pin suite (tests/test_oracle_pins.py) against it; the suite must fail.  The
mistakes are planted on the CPU, in the oracle only."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "leiden_oracle.c")

# (name, text in the oracle, replacement)
MUTANTS = [
    ("eq2_null_term_sign", "- (i128)p * Ki * (Ki + Sc - Sd)", "+ (i128)p * Ki * (Ki + Sc - Sd)"),
    ("eq2_dropped_Ki", "(Ki + Sc - Sd)", "(Sc - Sd)"),
    ("eq2_transposed_weights", "(Kic - Kid)", "(Kid - Kic)"),
    ("scan_counts_self_loop", "    if (j == i) continue;\n    if (CB && CB[j] != CB[i]) continue;",
     "    if (CB && CB[j] != CB[i]) continue;"),
    ("scan_ignores_bound", "    if (CB && CB[j] != CB[i]) continue;\n", ""),
    ("tie_to_largest_id", "(S == *Sbest && c < *cbest)", "(S == *Sbest && c > *cbest)"),
    ("move_on_zero_gain", "/* reading: move only to a strictly better community (S > 0) */\n        if (!found || Sbest <= 0)",
     "/* reading: move only to a strictly better community (S > 0) */\n        if (!found || Sbest < 0)"),
    ("eq1_gamma_on_wrong_side", "i128 num = (i128)q * two_m * sigma_in - (i128)p * sq;",
     "i128 num = (i128)p * two_m * sigma_in - (i128)q * sq;"),
    ("eq1_drops_self_loops", "if (C[idx[e]] == C[i]) sigma_in += w[e];",
     "if (C[idx[e]] == C[i] && idx[e] != i) sigma_in += w[e];"),
    ("aggregation_drops_internal_weight", "for (int64_t e = off[i]; e < off[i + 1]; e++) table_add(&t, C[idx[e]], w[e]);",
     "for (int64_t e = off[i]; e < off[i + 1]; e++) if (C[idx[e]] != c) table_add(&t, C[idx[e]], w[e]);"),
    ("subset_rep_is_largest", "if (rep[C[i]] < 0) rep[C[i]] = (int32_t)i;", "rep[C[i]] = (int32_t)i;"),
    ("break_reads_vertex_flag", "brk[i] = changed[C[i]];", "brk[i] = changed[i];"),
    ("refine_takes_non_isolated", "if (Sigma[c] != K[i]) continue; /* not isolated any more */", ""),
    ("update_weights_deletion_sign", "      K[i] -= dw[a];", "      K[i] += dw[a];"),
    ("changed_flag_of_vertex", "if (Cprev[ds[a]] == Cprev[dd[a]]) changed[Cprev[ds[a]]] = 1;",
     "if (Cprev[ds[a]] == Cprev[dd[a]]) changed[ds[a]] = 1;"),
    ("df_marks_cross_deletions", "if (Cprev[ds[a]] == Cprev[dd[a]]) { affected[ds[a]] = 1; affected[dd[a]] = 1; }",
     "if (Cprev[ds[a]] != Cprev[dd[a]]) { affected[ds[a]] = 1; affected[dd[a]] = 1; }"),
]


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, source, name, old, new):
    assert source.count(old) == 1, f"{name}: the planted spot must be unique"
    src = tmp_path / "mutant.c"
    src.write_text(source.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "oracle"), "-o", str(lib), str(src)])
    env = dict(os.environ, LEIDEN_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"{name}: the pins did not notice\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout, r.stdout[-2000:]
