"""The seeded input generators produce the shapes they state: the
differentiation batch's three kinds, sizes, strains and separations, and
the perturbed parameter set. No potential arithmetic is involved."""
import numpy as np
import pytest

from paper_1802_07871_gb300 import structures as st

P1 = st.load_params("p1")


@pytest.fixture(scope="module")
def batch():
    return st.differentiation_batch()


def _min_image_dist(s):
    d = s.x[:, None, :] - s.x[None, :, :]
    for a in range(3):
        if s.pbc[a]:
            d[..., a] -= np.round(d[..., a] / s.box[a]) * s.box[a]
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    np.fill_diagonal(r, np.inf)
    return r


def test_batch_sizes_and_kinds(batch):
    assert len(batch) == 1024
    n = np.array([s.n for s in batch])
    assert 280_000 < n.sum() < 310_000
    assert n.min() >= 60 and n.max() <= 520
    for c, s in enumerate(batch):
        assert s.name.startswith(("3C-SiC", "graphene", "random Si/C")[c % 3])


def test_strained_cells(batch):
    for s in batch[0::3][:60]:
        nc = np.array([int(v) for v in s.name.split()[1].split("x")])
        eps = s.box / (nc * 4.36) - 1.0
        assert np.all(np.abs(eps) <= 0.05 + 1e-12) and s.pbc.all()
        assert s.n == 8 * nc.prod() and np.sum(s.types == 0) == s.n // 2


def test_graphene_is_threefold(batch):
    for s in batch[1::3][:30]:
        r = _min_image_dist(s)
        assert np.all(np.sum(r < 1.7, axis=1) == 3)
        assert r.min() > 1.15 and np.all(s.types == 1)
        assert list(s.pbc) == [True, True, False]


def test_clusters_keep_their_separation(batch):
    for s in batch[2::3][:30]:
        r = _min_image_dist(s)
        assert r.min() >= 1.2 and not s.pbc.any()
        assert set(np.unique(s.types)) <= {0, 1}


def test_perturbed_params_change_only_stated_leaves():
    Pt = st.perturbed_params(P1, 55, rel=0.02)
    for name in P1["pair"]:
        for k, v in P1["pair"][name].items():
            if k in ("A", "B", "lambda1", "lambda2"):
                assert abs(Pt["pair"][name][k] / v - 1.0) <= 0.02 and Pt["pair"][name][k] != v
            else:
                assert Pt["pair"][name][k] == v
    for k in ("chi", "J"):
        for a, b in zip(Pt["self"][k], P1["self"][k]):
            assert abs(a / b - 1.0) <= 0.02
    assert Pt["self"]["E0"] == P1["self"]["E0"]
    assert Pt["triplet"] == P1["triplet"] and Pt["bond"] == P1["bond"] and Pt["coulomb"] == P1["coulomb"]


def test_sic_3c_cubic_unchanged_by_shape_argument():
    a, b = st.sic_3c(3, 4.36, 0.05, 9), st.sic_3c((3, 3, 3), 4.36, 0.05, 9)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.box, b.box)


def test_strain_generator_refuses_shear():
    """The differentiation batch strains its 3C-SiC cells along the cell axes
    only (the library's cells are orthorhombic): an off-diagonal strain is
    refused rather than silently dropped."""
    import pytest
    with pytest.raises(ValueError, match="orthorhombic"):
        st.sic_3c(2, 4.36, 0.0, strain=np.array([[0.01, 0.02, 0.0], [0.02, 0.0, 0.0], [0.0, 0.0, 0.0]]))
