"""The C-ABI library without a GPU: it loads, exports every entry point that
include/bsde.h declares, its struct layouts match the ctypes binding, and its
host-side basis builder matches the oracle.  CPU only (no compute calls)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bsde.h")


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    import paper_1102_4666_gb300 as G
    return G


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"BSDE_API\s+[\w\s\*]+?\b(bsde_\w+)\s*\(", text)))


def test_library_exports_every_declared_entry_point(G):
    names = declared_functions()
    assert len(names) >= 19
    L = ctypes.CDLL(G.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(G._SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", G.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == set(names)


C_LAYOUT = r"""
#include <stdio.h>
#include <stddef.h>
#include "bsde.h"
#define P(T) printf(#T " %zu\n", sizeof(T));
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  P(bsde_create_opts) O(bsde_create_opts, precision) O(bsde_create_opts, mem_budget)
  P(bsde_sigma) O(bsde_sigma, div) O(bsde_sigma, rho)
  P(bsde_payoff) O(bsde_payoff, weights)
  P(bsde_penalty) O(bsde_penalty, obstacle)
  P(bsde_solve_params) O(bsde_solve_params, seed) O(bsde_solve_params, allow_underdetermined) O(bsde_solve_params, eval_mode) O(bsde_solve_params, paths_ppt) O(bsde_solve_params, ls_mode) O(bsde_solve_params, gram_splits)
  P(bsde_report) O(bsde_report, ms_total) O(bsde_report, kernel_launches) O(bsde_report, resid_linf) O(bsde_report, rank)
  P(bsde_server_opts) O(bsde_server_opts, precision) O(bsde_server_opts, policy) O(bsde_server_opts, large_slots)
  P(bsde_request) O(bsde_request, params) O(bsde_request, hi) O(bsde_request, n)
  P(bsde_server_stats) O(bsde_server_stats, path_steps_per_s)
  P(bsde_peer_exchange) O(bsde_peer_exchange, flag) O(bsde_peer_exchange, c_len) O(bsde_peer_exchange, wait_ms) O(bsde_peer_exchange, pushed) O(bsde_peer_exchange, user)
  return 0;
}
"""


def test_struct_layouts_match_the_binding(G, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(C_LAYOUT)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        key, val = line.split()
        val = int(val)
        if "." in key:
            sname, field = key.split(".")
            cls = getattr(G, sname)
            field = "lambda_" if field == "lambda" else field
            assert getattr(cls, field).offset == val, key
        else:
            assert ctypes.sizeof(getattr(G, key)) == val, key


@pytest.mark.parametrize("d,eta,q", [(1, 4, 1.0), (1, 6, 1.0), (5, 4, 1.0), (10, 3, 1.0),
                                     (10, 5, 0.6), (5, 4, 0.75), (2, 0, 1.0), (3, 6, 0.5)])
def test_host_basis_matches_oracle(G, d, eta, q):
    from oracle import bsde_oracle as O
    nu = G.basis_indices(d, eta, q)
    ref = O.multi_index_set(d + 1, eta, q)
    assert nu.shape == ref.shape
    assert np.array_equal(nu, ref)


def test_host_validation_without_gpu(G):
    p = ctypes.c_int()
    assert G.lib().bsde_basis_size(0, 3, 1.0, ctypes.byref(p)) == G.ERR_INVALID_ARG
    assert G.lib().bsde_basis_size(3, 16, 1.0, ctypes.byref(p)) == G.ERR_INVALID_ARG
    assert G.lib().bsde_basis_size(3, 3, 1.5, ctypes.byref(p)) == G.ERR_INVALID_ARG
    assert G.lib().bsde_basis_size(6 - 1, 3, 1.0, ctypes.byref(p)) == G.OK and p.value == 84
    # NULL context is rejected without touching a device
    assert G.lib().bsde_solve(None, None, None) == G.ERR_INVALID_ARG
    assert G.lib().bsde_get_coeffs(None, None, 0) == G.ERR_INVALID_ARG
    assert G.lib().bsde_server_poll(None, 1, None) == G.ERR_INVALID_ARG
