"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

The paper prints no worked example (its Tables 1-3 are timings and its figures carry no
values), so these fixtures are regression anchors of the oracle on the small random-matrix
workload (GOE N=64, seeds 1/2, f = cos t, T = 2 pi, M = 200) and on a small dimer
(nb = 40, U nb/J = 2, eps1 = 1.5, omega = 3, M = 100).  Run:  python tests/golden/make_golden.py

`python tests/golden/make_golden.py adjoint1024` writes adjoint1024.txt: the oracle's loss and
gradient for the gate-fidelity workload at its own size (GOE N = 1024, seeds 6 and 7 for H0 and
H1, Haar target seed 8, f_m ~ N(1, 0.1^2) seed 9, M = 256 piecewise-constant steps, T = 2 pi,
bounds frozen from f as in reading R11).  It takes several minutes and about 5 GB of memory (the
oracle keeps every X_m), so it is a separate target.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import floquet_inputs as fi  # noqa: E402
import oracle as o  # noqa: E402


def goe64():
    m = fi.config_goe64()
    plan = o.plan_for_drive_dense(m.h0, m.h1, m.drive, m.steps)
    u = o.build_ut_dense(m.h0, m.h1, plan)
    return plan, u, o.quasienergies(u, m.drive.period)


def dimer40():
    d = fi.config_dimer(nb=40, steps=100)
    plan = o.plan_for_drive_tridiag(d.h0_diag, d.h0_off, d.h1_diag, d.drive, d.steps)
    u = o.build_ut_tridiag(d.h0_diag, d.h0_off, d.h1_diag, plan)
    return plan, u, o.quasienergies(u, d.drive.period)


def write(name, plan, u, eps):
    path = os.path.join(HERE, name)
    with open(path, "w") as fh:
        fh.write(f"# written by tests/golden/make_golden.py from oracle/ only\n")
        fh.write(f"R {float(plan.R)!r}\nL {plan.L}\n")
        fh.write(f"e_min {float(plan.e_min)!r}\ne_max {float(plan.e_max)!r}\n")
        for e in eps:
            fh.write(f"eps {float(e)!r}\n")
        n = u.shape[0]
        for i in range(0, n, max(1, n // 16)):
            for j in (0, i, n - 1):
                fh.write(f"u {i} {j} {float(u[i, j].real)!r} {float(u[i, j].imag)!r}\n")


def read(name):
    out = {"eps": [], "u": []}
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            k, *v = line.split()
            if k == "eps":
                out["eps"].append(float(v[0]))
            elif k == "u":
                out["u"].append((int(v[0]), int(v[1]), complex(float(v[2]), float(v[3]))))
            else:
                out[k] = float(v[0])
    return out


def adjoint1024():
    import math
    n, steps = 1024, 256
    h0, h1 = fi.goe(n, 6), fi.goe(n, 7)
    w = fi.haar_unitary(n, 8)
    fm = 1.0 + 0.1 * fi.normal(9, steps)
    plan = o.plan_piecewise(h0, h1, 2 * math.pi, fm)
    loss, grad = o.grad_piecewise(h0, h1, w, plan, fm)
    return plan, loss, grad


def write_adjoint(name, plan, loss, grad):
    with open(os.path.join(HERE, name), "w") as fh:
        fh.write("# written by tests/golden/make_golden.py adjoint1024 from oracle/ only\n")
        fh.write(f"R {float(plan.R)!r}\nL {plan.L}\n")
        fh.write(f"beta {float(plan.beta)!r}\ndelta_e {float(plan.delta_e)!r}\n")
        fh.write(f"loss {float(loss)!r}\n")
        for m, g in enumerate(grad):
            fh.write(f"g {m} {float(g)!r}\n")


def read_adjoint(name):
    out = {"g": []}
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            k, *v = line.split()
            if k == "g":
                out["g"].append(float(v[1]))
            else:
                out[k] = float(v[0])
    return out


if __name__ == "__main__":
    if sys.argv[1:] == ["adjoint1024"]:
        write_adjoint("adjoint1024.txt", *adjoint1024())
    else:
        write("goe64.txt", *goe64())
        write("dimer40.txt", *dimer40())
    print("written")
