"""The oracle's pins catch plausible mistakes.

Each case copies oracle/oracle.c, plants one mistake in the copy (a
transposed operand, a wrong stride, a wrong tuple enumeration, a dropped
factor), builds it with gcc and runs the pins of test_oracle_pins.py against
that build: at least one pin must fail.  Nothing here touches the GPU
library.
"""
import subprocess
from pathlib import Path

import pytest

import oracle
import test_oracle_pins as pins

SRC = Path(oracle.__file__).resolve().parent / "oracle.c"

# (name, text in oracle.c, planted replacement)
MUTATIONS = [
    ("brute force reads X transposed", "prod *= X[j[k] + ik * p];", "prod *= X[ik + j[k] * n];"),
    ("mode product reads X transposed", "double bji = B[j + i * q];", "double bji = B[i + j * nk];"),
    ("mode product with a wrong input stride", "const double* src = in + left * (i + nk * r);",
     "const double* src = in + left * (i * right + r);"),
    ("entry contraction reads X transposed", "double x = X[j[k] + i * p];", "double x = X[j[k] * n + i];"),
    ("block tuples not restricted to sorted ones", "int64_t upper = (a + 1 < m) ? t[a + 1] : nbar - 1;",
     "int64_t upper = nbar - 1;"),
    # (counted one too many: the wrapper allocates by the count, so the
    # planted error never makes the C code write past the buffer)
    ("block count off by one", "int64_t count = 1;", "int64_t count = 2;"),
    ("flop count drops the factor 2", "double per = 2.0 * (double)ipow(bC, d + 1)",
     "double per = 1.0 * (double)ipow(bC, d + 1)"),
    ("flop count with a wrong C-block exponent", "(double)ipow(bC, d + 1) * (double)ipow(bA, m - d)",
     "(double)ipow(bC, d) * (double)ipow(bA, m - d)"),
]

# pins run against each mutant (cheap ones; each a zero-argument call)
PINS = [
    ("bruteforce rank-r", lambda: pins.test_bruteforce_rank_r_closed_form(2, 4, 6, 1)),
    ("bruteforce m=2", pins.test_bruteforce_m2_is_X_A_Xt),
    ("bruteforce special matrices", pins.test_bruteforce_special_matrices),
    ("chain per-mode einsum", pins.test_chain_per_mode_matrices_match_einsum),
    ("chain vs bruteforce", lambda: pins.test_chain_equals_bruteforce(3, 5, 7)),
    ("chain rank-2 closed form", pins.test_chain_rank2_config1_closed_form),
    ("entries vs chain", pins.test_entries_equal_chain),
    ("paper's m=2 order", pins.test_bcss_b1_m2_order_matches_paper_picture),
    ("block count", lambda: pins.test_bcss_block_count_is_binomial(3)),
    ("pack blocks", lambda: pins.test_bcss_pack_blocks_and_padding(3, 10, 4)),
    ("flops vs Tbl. 4", lambda: pins.test_flop_count_matches_mincosts_table(3, 24, 24, 8)),
    ("flops b=1 identity", lambda: pins.test_flop_count_b1_exact_identity(3, 6)),
]


def test_unmutated_copy_passes_every_pin(tmp_path):
    so = tmp_path / "liboracle_copy.so"
    (tmp_path / "oracle.c").write_text(SRC.read_text())
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", str(tmp_path / "oracle.c"),
                    "-o", str(so), "-lm"], check=True)
    with oracle.library(so):
        for _, pin in PINS:
            pin()


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    text = SRC.read_text()
    assert text.count(old) == 1, "mutation site not found: " + old
    src = tmp_path / "oracle.c"
    src.write_text(text.replace(old, new))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", str(src), "-o", str(so),
                    "-lm"], check=True)
    failed = []
    with oracle.library(so):
        for pin_name, pin in PINS:
            try:
                pin()
            except (AssertionError, IndexError, ValueError):
                failed.append(pin_name)
    assert failed, "no pin caught: " + name
