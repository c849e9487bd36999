"""Pins of the seeded input recipe (floquet_inputs), which both the CUDA path and the oracle
consume: the counter generator against its published outputs, the distributions against their
textbook moments, and the dimer's Fock-basis matrices against a brute-force construction from
the two modes' ladder operators."""
import math

import numpy as np
from scipy import stats

import floquet_inputs as fi


def test_splitmix64_published_outputs():
    """The first outputs of splitmix64 seeded with 0, as published with the generator."""
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [int(x) for x in fi.splitmix64(0, 5)] == ref
    # the counter form: outputs k+1.. of a stream equal the tail of a longer draw
    assert np.array_equal(fi.splitmix64(7, 3, offset=10), fi.splitmix64(7, 13)[10:])


def test_uniform_and_normal_distributions():
    u = fi.uniform(11, 200_000)
    assert np.all((u > 0) & (u < 1))
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    z = fi.normal(12, 200_000)
    assert abs(np.mean(z)) < 0.01 and abs(np.var(z) - 1) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # odd lengths are a prefix of the next even draw
    assert np.array_equal(fi.normal(5, 7), fi.normal(5, 8)[:7])


def test_goe_normalisation_and_semicircle():
    """(G + G^T)/sqrt(2N): symmetric, off-diagonal variance 1/N, diagonal variance 2/N, and the
    spectrum fills the semicircle on [-2, 2]."""
    n = 800
    h = fi.goe(n, 21)
    assert np.array_equal(h, h.T) and h.flags.c_contiguous
    off = h[np.triu_indices(n, 1)]
    assert abs(np.var(off) * n - 1) < 0.02
    assert abs(np.var(np.diag(h)) * n / 2 - 1) < 0.15
    ev = np.linalg.eigvalsh(h)
    assert abs(ev[-1] - 2) < 0.1 and abs(ev[0] + 2) < 0.1
    # second moment of the semicircle of radius 2 is 1
    assert abs(np.mean(ev ** 2) - 1) < 0.02
    assert not np.array_equal(fi.goe(n, 21), fi.goe(n, 22))


def test_haar_unitary():
    """Unitary, and |U_11|^2 has the Beta(1, n - 1) mean 1/n of a Haar column entry; the
    eigenphases have no preferred direction (mean resultant length ~ 1/sqrt(n))."""
    n = 64
    us = [fi.haar_unitary(n, 100 + s) for s in range(200)]
    for u in us[:5]:
        assert np.max(np.abs(u.conj().T @ u - np.eye(n))) < 1e-13
    p = np.array([abs(u[0, 0]) ** 2 for u in us])
    assert abs(np.mean(p) * n - 1) < 0.2
    ph = np.concatenate([np.angle(np.linalg.eigvals(u)) for u in us[:20]])
    assert abs(np.mean(np.exp(1j * ph))) < 5 / math.sqrt(ph.size)


def _two_mode_dimer(nb, J, U, paper):
    """Brute force: truncated ladder operators of two modes, the Hamiltonian on the full
    (nb+1)^2 space, then the block of total number nb in the basis |n, nb - n>."""
    d = nb + 1
    a = np.diag(np.sqrt(np.arange(1, d)), 1)       # a|k> = sqrt(k)|k-1>
    eye = np.eye(d)
    a1, a2 = np.kron(a, eye), np.kron(eye, a)
    n1, n2 = a1.T @ a1, a2.T @ a2
    hop = a1.T @ a2 + a2.T @ a1
    if paper:
        h0 = -J * hop + 0.5 * U * (n1 - n2) @ (n1 - n2)
        h1 = n2 - n1
    else:
        h0 = -J * hop + 0.5 * U * (n1 @ (n1 - np.eye(d * d)) + n2 @ (n2 - np.eye(d * d)))
        h1 = 0.5 * (n1 - n2)
    idx = [n * d + (nb - n) for n in range(nb + 1)]  # |n1 = n, n2 = nb - n>
    return h0[np.ix_(idx, idx)], h1[np.ix_(idx, idx)]


def test_dimer_matrices_against_ladder_operators():
    for nb, J, U in ((1, 1.0, 0.3), (6, 1.0, 0.25), (9, 0.7, 0.1)):
        for paper in (False, True):
            h0, h1 = _two_mode_dimer(nb, J, U, paper)
            if paper:
                dd, off, h1d = fi.dimer_matrices_paper(nb, v=J, U=U)
            else:
                dd, off, h1d = fi.dimer_matrices(nb, J=J, U=U)
            ref0 = np.diag(dd) + np.diag(off, -1) + np.diag(off, 1)
            assert np.max(np.abs(h0 - ref0)) < 1e-12, (nb, paper)
            assert np.max(np.abs(h1 - np.diag(h1d))) < 1e-12, (nb, paper)
    # defaults: U nb / J = 2 (this form) and U nb = 2 (the paper's form)
    dd, _, _ = fi.dimer_matrices(10, J=1.0)
    assert abs(dd[0] - 0.5 * (2.0 / 10) * 10 * 9) < 1e-12
    dd, _, _ = fi.dimer_matrices_paper(10)
    assert abs(dd[0] - 0.5 * (2.0 / 10) * 100) < 1e-12


def test_batch_scan_ranges_and_seeds():
    insts = fi.batch_scan()
    assert len(insts) == 48
    assert all(256 <= s.n <= 2048 for s in insts)
    assert all(0.5 <= s.omega <= 4.0 and 0.5 <= s.amplitude <= 3.0 for s in insts)
    seeds = [s.seed_h0 for s in insts] + [s.seed_h1 for s in insts]
    assert len(set(seeds)) == len(seeds)
    assert insts == fi.batch_scan()  # deterministic
