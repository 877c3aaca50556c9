"""The pins are sharp enough to catch a plausible mistake: copies of the
oracle's C source, each with one mistake planted (a dropped factor, a sign,
a missing renormalisation, q and tau swapped, a skewed label law, a biased
rule for odd counts, lowering the depth where leaves can be borrowed, a
wall that forgets to reverse v_x, a permutation with too few rounds or a
Feistel network on domains too small for one), are built into their own libraries and run
through the pins of tests/test_oracle_*.py; every copy must fail at least
one of them.  The oracle itself is untouched: the copies live in a
temporary directory and the module is pointed back at the real library
afterwards."""
import os
import shutil
import subprocess

import pytest

from oracle import oracle as O
from tests import test_oracle_euler_limit as E
from tests import test_oracle_physics as P
from tests import test_oracle_plan_law as PL
from tests import test_oracle_rng as RNG
from tests import test_oracle_transport_init as TI

ORACLE_DIR = os.path.dirname(os.path.abspath(O.__file__))
SOURCES = ["rng.c", "collide.c", "transport.c", "init_moments.c"]

MISTAKES = {
    "collision: the half of the relative speed dropped":
        ("collide.c", "double h = 0.5 * g;", "double h = g;"),
    "collision: the second product's sign flipped":
        ("collide.c", "ob->x = cx - h * sx; ob->y = cy - h * sy; ob->z = cz - h * sz;",
         "ob->x = cx + h * sx; ob->y = cy + h * sy; ob->z = cz + h * sz;"),
    "Maxwellian: no renormalisation":
        ("collide.c", "double s = (ez > 0.0) ? sqrt(et / ez) : 0.0;", "double s = (ez > 0.0) ? 1.0 : 0.0;"),
    "split: tau where q belongs":
        ("collide.c", "double q = exp(-(mu * dt) / eps);", "double q = -expm1(-(mu * dt) / eps);"),
    "labels: k drawn from the lower half only":
        ("collide.c", "lab[c] = (int32_t)orc_below(w[c & 3], (uint32_t)n);",
         "lab[c] = (int32_t)orc_below(w[c & 3], (uint32_t)(n + 1) / 2);"),
    "odd count: the surplus product always kept (always round up)":
        ("collide.c", "if (pl->Nn[n] >= 1 && orc_u01(w[0]) < 0.5)", "if (0 && pl->Nn[n] >= 1 && orc_u01(w[0]) < 0.5)"),
    "odd count: a quota particle always dropped when the level has one":
        ("collide.c", "if (pl->Nn[n] >= 1 && orc_u01(w[0]) < 0.5)", "if (pl->Nn[n] >= 1)"),
    "leaves: the depth lowered instead of borrowing from level 0":
        ("collide.c", "if (deficit <= n0) {", "if (0) {"),
    "permutation: four Feistel rounds":
        ("rng.c", "    return p->b <= 8 ? 8 : 6;", "    return 4;"),
    "permutation: five Feistel rounds on words wider than 8 bits":
        ("rng.c", "    return p->b <= 8 ? 8 : 6;", "    return p->b <= 8 ? 8 : 5;"),
    "permutation: the Feistel network for cells of up to 32 items too":
        ("rng.c", "    if (p->n <= 32) {\n        uint32_t kx", "    if (0) {\n        uint32_t kx"),
    "walls: the right wall keeps v_x":
        ("transport.c", "else if (xn > hi) { xn = 2.0 * hi - xn; vx[i] = -vx[i]; }",
         "else if (xn > hi) { xn = 2.0 * hi - xn; }"),
}

# cheap pins first; a copy stops at the first pin it fails
PINS = [
    ("transport hand example", TI.test_transport_hand_example),
    ("permutation: top ranks of 5 items", lambda: RNG.test_prp_top_ranks_form_a_uniform_subset(5)),
    ("permutation: top ranks of 33 items", lambda: RNG.test_prp_top_ranks_form_a_uniform_subset(33)),
    ("permutation: top ranks in a block of 500", lambda: RNG.test_prp_top_ranks_in_a_block_are_hypergeometric(500, 12000)),
    ("permutation: fixed points of 300 items", lambda: RNG.test_prp_fixed_points_are_poisson(300, 30000)),
    ("conservation, hard spheres, TRMC-RAD", lambda: P.test_conservation(1.0, 0.05, O.TRUNC_RAD, 2)),
    ("conservation, Maxwell molecules, eps 1e-4", lambda: P.test_conservation(0.0, 1e-4, O.TRUNC_FIXED, 1)),
    ("level occupation", P.test_level_occupation_expectation),
    ("tree label law", P.test_tree_label_law),
    ("plan law by enumeration, 6 particles, m = 3", lambda: PL.test_oracle_plan_follows_the_enumerated_law(6, 3, 0.7)),
    ("plan law by enumeration, 4 particles, m = 3", lambda: PL.test_oracle_plan_follows_the_enumerated_law(4, 3, 1.6)),
    ("outputs unbiased per level", lambda: PL.test_outputs_are_unbiased_per_level(0.7)),
    ("M4 step factor, m = 2", lambda: P.test_m4_step_factor_maxwell(2)),
    ("Euler limit of the shock tube", E.test_oracle_shock_tube_follows_the_euler_riemann_solution),
]


def build_copy(tmp, name, fname, old, new):
    d = os.path.join(tmp, name.split(":")[0].replace(" ", "_") + str(abs(hash(name)) % 10000))
    os.makedirs(d)
    for f in SOURCES + ["trmc_oracle.h"]:
        shutil.copy(os.path.join(ORACLE_DIR, f), d)
    path = os.path.join(d, fname)
    src = open(path).read()
    assert src.count(old) == 1, f"the text to change is not unique in {fname}: {old}"
    open(path, "w").write(src.replace(old, new))
    lib = os.path.join(d, "liborc_copy.so")
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    "-pthread", "-o", lib] + [os.path.join(d, s) for s in SOURCES] + ["-lm"], check=True)
    return lib


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_every_planted_mistake_fails_a_pin(name, tmp_path, monkeypatch):
    lib = build_copy(str(tmp_path), name, *MISTAKES[name])
    monkeypatch.setattr(O, "build_oracle", lambda force=False: lib)
    monkeypatch.setattr(O, "_lib", None)
    caught = None
    for pin, run in PINS:
        try:
            run()
        except AssertionError:
            caught = pin
            break
    assert caught is not None, f"no pin fails with the planted mistake '{name}'"


def test_the_unchanged_oracle_passes_the_same_pins():
    for pin, run in PINS:
        run()
