"""Write the oracle regression fixtures in this directory.

Calls only the oracle (and the input generators). The stored numbers are the
oracle's own outputs on small seeded cases; the tests check that later
changes to the oracle leave them unchanged (to 1e-9 relative: libm may differ
in the last bit between machines).

Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def heat65_case(exit_mode):
    xi0, eta0 = W.heat65_fields()
    P = oracle.Problem(W.w_const(65), xi0, eta0, np.zeros(oracle.faces_len(65, 65)))
    xs, ys = W.heat65_nodes()
    r = oracle.interface_mc(P, xs, ys, 1000, dt=1e-3, Dt=0.05, seed=0, exit_mode=exit_mode)
    return {k: np.asarray(v).tolist() for k, v in r.items()}


def front_case():
    n = 65
    xi0, eta0 = W.identity_fields(n)
    P = oracle.Problem(W.w_front(n, 0.1), xi0, eta0)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    sel = np.arange(0, xs.size, 9)
    r = oracle.interface_mc(P, xs[sel], ys[sel], 500, dt=1e-4, Dt=1e-2, seed=7, exit_mode=0, step_index=3,
                            node_ids=sel.astype(np.uint32))
    return {k: np.asarray(v).tolist() for k, v in r.items()}


def front_cell_cv_case():
    # the field-gradient control variate as cell values (order 5) on fields with structure
    from oracle import mlp
    n = 65
    X, Y = W.grid(n)
    xi0 = X + 0.02 * np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
    eta0 = Y + 0.01 * np.sin(3 * np.pi * X) * np.sin(np.pi * Y)
    P = oracle.Problem(W.w_front(n, 0.1), xi0, eta0)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    sel = np.arange(0, xs.size, 11)
    r = oracle.interface_mc(P, xs[sel], ys[sel], 500, dt=1e-4, Dt=1e-2, seed=9, exit_mode=0, step_index=2,
                            cv_table=mlp.field_cell_gradient_table(xi0, eta0, 5))
    return {k: np.asarray(v).tolist() for k, v in r.items()}


def main():
    out = {
        "about": "oracle outputs on small seeded cases; written by tests/golden/make_golden.py",
        "heat65_plain": heat65_case(0),
        "heat65_bridge": heat65_case(1),
        "front65_plain": front_case(),
        "front65_cell_cv": front_cell_cv_case(),
    }
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
