"""Pins of the oracle's per-stencil condition numbers (Section 2.1)."""
import numpy as np

from oracle import stencils as ost
from oracle import weights as ow
from paper_2303_01760_gb300 import nodesets


def test_mon_lattice_stencil_closed_form():
    """The scaled 5-point MON matrix (offsets 0, +-e1, +-e2) has Gram matrix
    eigenvalues 2, 2, 2 and (7 +- sqrt 41)/2, so kappa_2 = (7 + sqrt 41) / (2 sqrt 2)."""
    coords = np.array([[0.0, -1.0, 1.0, 0.0, 0.0], [0.0, 0.0, 0.0, -1.0, 1.0]]) * 0.37 + 0.5
    st = {"mon_idx": np.array([[0, 1, 2, 3, 4]]), "rbf_idx": np.zeros((0, 12), dtype=np.int64)}
    k = ow.condition_numbers(coords, st, 2)["mon"]
    assert abs(k[0] - (7 + np.sqrt(41)) / (2 * np.sqrt(2))) <= 1e-12


def test_rbf_condition_from_the_spectrum():
    """The augmented RBF-FD matrix is symmetric, so kappa_2 is the ratio of its
    largest and smallest eigenvalue magnitudes (an independent route)."""
    ns = nodesets.square_wall_band(n=24)
    st = ost.build_stencils(ns.coords, ns.is_regular, ns.is_boundary, ns.h, 12, normals=ns.normals)
    k = ow.condition_numbers(ns.coords, st, 2)
    xi, _ = ow._scaled_offsets(ns.coords, st["rbf_idx"])
    M, _ = ow.rbffd_system(xi, 2, ow.ops_for(2))
    lam = np.abs(np.linalg.eigvalsh(M))
    assert np.allclose(k["rbf"], lam.max(1) / lam.min(1), rtol=1e-9)
    # the qualitative claim of Section 2.1: RBF-FD systems are worse conditioned
    assert np.median(k["rbf"]) > 10 * np.median(k["mon"])
    assert np.all(k["mon"] >= 1.0)
