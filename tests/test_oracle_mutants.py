"""The oracle's pins reject plausible mistakes.

Each case copies the oracle's C source, plants one mistake of the kind a
restatement of the paper could make (a dropped random word, a wrong key, a
flipped comparison), builds the copy, and runs the pin that should catch it
against that copy in a fresh interpreter.  The pin must fail.  The committed
oracle is never modified; the copies live in pytest's temporary directory.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "pamc_oracle.c")

PINS = "tests/test_oracle_pins_init_ncm.py"

# (name, text in the oracle, planted replacement, pin that must fail)
MUTANTS = [
    ("constant initial spins",
     "if (st->p.kind == 0) v = (x >> 31) ? 1 : -1;",
     "if (st->p.kind == 0) v = 1;",
     PINS + "::test_initial_ising_population_uniform_and_independent"),
    ("one random word for every replica of a call",
     "uint32_t x = u[r & 3];",
     "uint32_t x = u[0];",
     PINS + "::test_initial_ising_population_uniform_and_independent"),
    ("initial draws keyed by site pairs",
     "orc_draw4(st->p.seed, (uint32_t)i, 0u, (uint32_t)t,",
     "orc_draw4(st->p.seed, (uint32_t)(i >> 1), 0u, (uint32_t)t,",
     PINS + "::test_initial_ising_population_uniform_and_independent"),
    ("restart re-draws with the first key",
     "orc_init_population(st, st->t + 1);",
     "orc_init_population(st, 0);",
     PINS + "::test_restart_redraws_an_independent_population"),
    ("restart keeps the population",
     "if (restart && st->p.restart_reinit)",
     "if (restart && st->p.restart_reinit && 0)",
     PINS + "::test_restart_redraws_an_independent_population"),
    ("cluster move on the highest-energy replicas",
     "return orc_sort_E[x] < orc_sort_E[y] ? -1 : 1;",
     "return orc_sort_E[x] < orc_sort_E[y] ? 1 : -1;",
     PINS + "::test_ncm_targets_are_the_lowest_energy_replicas_ties_to_lower_slot"),
    ("cluster-move ties to the higher slot",
     "return x < y ? -1 : (x > y ? 1 : 0);",
     "return x < y ? 1 : (x > y ? -1 : 0);",
     PINS + "::test_ncm_targets_are_the_lowest_energy_replicas_ties_to_lower_slot"),
]


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_rejects_planted_mistake(tmp_path, name, old, new, pin):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old}"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-I", os.path.join(ROOT, "oracle"), "-o", str(lib), str(mutant), "-lm"])
    env = dict(os.environ, PAMC_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", pin, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"{name}: the pin passed on the mutant\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout
