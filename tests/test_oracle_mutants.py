"""Mutation check of the pins: plausible slips planted in a COPY of the oracle (on the CPU)
must each be caught by at least one of the pins P1-P9."""
import os
import subprocess

import pytest

import oracle
import pin_suite

MUTANTS = {
    # the paper's inclusive side test (Algorithm 1 counts line_pos <= 0)
    "inclusive-side": ("if (line_pos < 0)", "if (line_pos <= 0)"),
    # the opposite half-open convention (a vertex on the ray counted as above)
    "flip-half-open": ("if ((f_i > 0) == (f_j > 0))", "if ((f_i >= 0) == (f_j >= 0))"),
    # the paper's sign-change product read literally (f_i f_{i+1} <= 0)
    "literal-sign-change": ("if ((f_i > 0) == (f_j > 0))", "if (f_i * f_j > 0)"),
    # a dropped term of the dot product
    "dropped-term": (" + (i128)(py - y_i) * n_y;", ";"),
    # a wrong sign in the normal's orientation
    "wrong-flip": ("if (n_x < 0) {", "if (n_x > 0) {"),
    # transposed operands in the normal
    "transposed-normal": ("int64_t n_x = d_y, n_y = -d_x;", "int64_t n_x = d_x, n_y = -d_y;"),
    # a wrong index: the closing edge R_{m-1} -> R_0 dropped
    "no-closing-edge": ("int64_t j = (i + 1 == m) ? 0 : i + 1;", "int64_t j = (i + 1 == m) ? i : i + 1;"),
    # products formed in 64 bits (overflow at the full int32 range)
    "int64-product": ("(i128)(px - x_i) * n_x + (i128)(py - y_i) * n_y",
                      "(i128)((px - x_i) * n_x + (py - y_i) * n_y)"),
    # f computed against the wrong coordinate
    "f-uses-x": ("int64_t f_i = y_i - py;", "int64_t f_i = x_i - px;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    before, after = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(before) == 1, f"mutation anchor for {name} not found exactly once"
    mut = src.replace(before, after)
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(mut)
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC", "-pthread",
                           "-o", str(so), str(c)])
    lib = oracle.open_library(str(so))
    caught = []
    for pin in pin_suite.ALL_PINS:
        if pin(lib):
            caught.append(pin.__name__)
            break
    assert caught, f"mutant {name} passed every pin"
