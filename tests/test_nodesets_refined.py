"""The h-refined node sets of Sections 4.2 and 4.3: the internodal distance
falls linearly from h_r (regular nodes) to h_s = h_r/ratio on the obstacles
over a distance h_r * delta_h, which is also the width of the scattered
layer.  Input data only: these check the generator, not the method."""
import numpy as np
from scipy.spatial import cKDTree

from paper_2303_01760_gb300 import nodesets


def _gap(ns):
    c = ns.holes[:, :ns.dim]
    r = ns.holes[:, ns.dim]
    return (np.sqrt(((ns.coords.T[:, None, :] - c[None]) ** 2).sum(-1)) - r[None]).min(1)


def test_spacing_function_and_layer_width():
    ns = nodesets.holes_refined(n=40, n_holes=2, r_range=(0.1, 0.15), delta_h=4.0, seed=nodesets.SEED_BASE + 60)
    h_r, h_s = ns.h, ns.h / 3.0
    g = _gap(ns)
    expect = h_s + (h_r - h_s) * np.clip(g / (4.0 * h_r), 0.0, 1.0)
    on_hole = (ns.is_boundary == 1) & (ns.bc == nodesets.BC_T_DIRICHLET)
    on_box = (ns.is_boundary == 1) & ~on_hole
    fill = (ns.is_regular == 0) & (ns.is_boundary == 0)
    # fill nodes carry h(x); hole nodes h_s; lattice and box-wall nodes h_r
    assert np.allclose(ns.spacing[fill], expect[fill], rtol=0, atol=1e-15)
    assert np.allclose(ns.spacing[on_hole], h_s)
    assert np.all(ns.spacing[(ns.is_regular == 1) | on_box] == h_r)
    # every regular node lies outside the layer, every scattered interior node inside it
    assert np.all(g[ns.is_regular == 1] >= 4.0 * h_r - 1e-9 * h_r)
    scat = (ns.is_regular == 0) & (ns.is_boundary == 0)
    assert np.all(g[scat] < 4.0 * h_r + 1e-12)
    # nearest-neighbour distances follow the local spacing; no fill node is
    # closer to another node than the larger of their two spacings
    tree = cKDTree(ns.coords.T)
    d, _ = tree.query(ns.coords.T, k=2)
    ratio = d[:, 1] / ns.spacing
    assert ratio[scat].min() > 0.8
    assert np.median(ratio[scat]) < 1.3
    pairs = tree.query_pairs(h_r * (1 - 1e-9), output_type="ndarray")
    i, j = pairs[:, 0], pairs[:, 1]
    dd = np.sqrt(((ns.coords[:, i] - ns.coords[:, j]) ** 2).sum(0))
    either_fill = fill[i] | fill[j]
    assert np.all(dd[either_fill] >= np.maximum(ns.spacing[i], ns.spacing[j])[either_fill] * (1 - 1e-9))


def test_layer_width_sweep_and_fully_scattered():
    """A wider layer (larger delta_h) holds more scattered nodes; the fully
    scattered set has no regular node and the same spacing at the holes."""
    sets = [nodesets.holes_refined(n=40, n_holes=2, r_range=(0.1, 0.15), delta_h=d, seed=nodesets.SEED_BASE + 60)
            for d in (2.0, 4.0, 8.0)]
    ns_ = [s.n_scattered for s in sets]
    assert ns_[0] < ns_[1] < ns_[2]
    full = nodesets.holes_refined(n=40, n_holes=2, r_range=(0.1, 0.15), delta_h=4.0, all_scattered=True,
                                  seed=nodesets.SEED_BASE + 60)
    assert int(full.is_regular.sum()) == 0
    assert np.array_equal(full.holes, sets[1].holes)
    assert full.spacing.min() == sets[1].spacing.min()


def test_refined_3d_and_cache_roundtrip(tmp_path):
    ns = nodesets.holes_refined(dim=3, n=12, n_holes=1, r_range=(0.15, 0.2), delta_h=3.0, ratio=2.0,
                                seed=nodesets.SEED_BASE + 61)
    assert ns.dim == 3 and ns.spacing.shape == (ns.N,)
    assert np.isclose(ns.spacing.min(), ns.h / 2.0)
    a = nodesets.cached(nodesets.holes_refined, dim=3, n=12, n_holes=1, r_range=(0.15, 0.2), delta_h=3.0,
                        ratio=2.0, seed=nodesets.SEED_BASE + 61, cache_dir=str(tmp_path))
    b = nodesets.cached(nodesets.holes_refined, dim=3, n=12, n_holes=1, r_range=(0.15, 0.2), delta_h=3.0,
                        ratio=2.0, seed=nodesets.SEED_BASE + 61, cache_dir=str(tmp_path))
    assert np.array_equal(a.coords, ns.coords) and np.array_equal(b.spacing, ns.spacing)
    plain = nodesets.cached(nodesets.square_wall_band, n=10, cache_dir=str(tmp_path))
    assert nodesets.cached(nodesets.square_wall_band, n=10, cache_dir=str(tmp_path)).spacing is None
    assert plain.spacing is None


def test_fill_keeps_clear_of_the_box_faces():
    """Fill nodes keep half a local spacing from every box face, so none sits
    in the empty channel along a 3D box edge (whose lattice nodes are dropped)."""
    for ns in (nodesets.holes_refined(n=40, n_holes=2, r_range=(0.1, 0.15), delta_h=4.0, all_scattered=True,
                                      seed=nodesets.SEED_BASE + 60),
               nodesets.holes_refined(dim=3, n=12, n_holes=1, r_range=(0.15, 0.2), delta_h=3.0, ratio=2.0,
                                      all_scattered=True, seed=nodesets.SEED_BASE + 61)):
        fill = (ns.is_regular == 0) & (ns.is_boundary == 0)
        face = np.minimum(ns.coords, 1.0 - ns.coords).min(0)
        assert np.all(face[fill] >= 0.5 * ns.spacing[fill] * (1 - 1e-12))
