"""GPU parity: geometry, visibility, insolation and partition of libvf
against the oracle (integer outputs bit-exact; floats to FP64 rounding)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_07632_gb300 import vf as _vf
    return _vf


def _meshes():
    out = dict(synth.tiny_meshes())
    out["bowl_small"] = synth.cap_bowl_mesh(n_rim=24, n_interior=90, seed=3)
    out["dem12"] = synth.fbm_dem_mesh(n=12, spacing=10.0, seed=9, crater_diameter=60.0)
    out["sphere2"] = synth.gaussian_sphere_mesh(level=2, sigma=0.3, seed=2)
    return out


MESHES = _meshes()


@pytest.mark.parametrize("name", sorted(MESHES))
def test_geometry_matches_oracle(vf, name):
    v, f = MESHES[name]
    m = vf.vf_mesh_create(v, f)
    om = oracle.mesh(v, f)
    unit, base = vf.vf_mesh_grid(m)
    assert unit == om.unit and np.array_equal(base, om.base)
    area, cent, nrm = vf.vf_mesh_geometry(m)
    assert np.allclose(area, om.area, rtol=1e-13, atol=0)
    assert np.allclose(cent, om.cent, rtol=1e-13, atol=1e-15 * np.abs(om.cent).max())
    assert np.allclose(nrm, om.nrm, rtol=0, atol=1e-13)


@pytest.mark.parametrize("name", sorted(MESHES))
def test_visibility_bit_exact_vs_brute_force(vf, name):
    v, f = MESHES[name]
    m = vf.vf_mesh_create(v, f)
    Vg = vf.vf_mesh_visibility(m)
    Vo = oracle.visibility_brute(oracle.mesh(v, f))
    assert np.array_equal(Vg, Vo)


def test_visibility_cap_full_bit_exact(vf, cap_full_F):
    v, f = synth.cap_bowl_mesh()
    m = vf.vf_mesh_create(v, f)
    assert np.array_equal(vf.vf_mesh_visibility(m), cap_full_F[1])


def test_visibility_sampled_rows_full_size_dem(vf):
    """The 79,202-facet terrain: sampled rows bit-exact vs the oracle BVH."""
    v, f = synth.fbm_dem_mesh()
    m = vf.vf_mesh_create(v, f)
    om = oracle.mesh(v, f)
    rows = np.random.default_rng(7).choice(om.n, size=6, replace=False)
    assert np.array_equal(vf.vf_mesh_visibility(m, rows), oracle.visibility_rows(om, rows))


@pytest.mark.parametrize("name", ["bowl_small", "dem12", "sphere2", "open_box"])
def test_insolation_matches_oracle(vf, name):
    import torch
    v, f = MESHES[name]
    m = vf.vf_mesh_create(v, f)
    om = oracle.mesh(v, f)
    dirs = np.concatenate([synth.sun_directions(5, 20.0), synth.sun_directions(2, -10.0)])
    E = torch.empty((dirs.shape[0], om.n), device="cuda")
    vf.vf_mesh_insolation(m, dirs, 1365.0, E)
    Eg = E.double().cpu().numpy().T
    Eo = oracle.insolation(om, dirs, 1365.0, brute=True)
    assert np.array_equal(Eg > 0, Eo > 0)
    assert np.allclose(Eg, Eo, rtol=1e-6, atol=1e-4)


def test_insolation_cap_shadow(vf, cap_full):
    import torch
    v, f = synth.cap_bowl_mesh()
    m = vf.vf_mesh_create(v, f)
    s = synth.sun_directions(3, 10.0)
    E = torch.empty((3, cap_full.n), device="cuda")
    vf.vf_mesh_insolation(m, s, 1365.0, E)
    Eo = oracle.insolation(cap_full, s, 1365.0)
    assert np.array_equal(E.cpu().numpy().T > 0, Eo > 0)


@pytest.mark.parametrize("kind,mesh,leaf", [("quad", "dem", 16), ("quad", "cap", 64), ("oct", "sphere", 20),
                                            ("quad", "tiny", 1)])
def test_partition_bit_exact(vf, kind, mesh, leaf):
    if mesh == "dem":
        v, f = synth.fbm_dem_mesh(n=30, seed=3, crater_diameter=120.0)
    elif mesh == "cap":
        v, f = synth.cap_bowl_mesh()
    elif mesh == "sphere":
        v, f = synth.gaussian_sphere_mesh(level=3, seed=4)
    else:
        v, f = synth.tiny_meshes()["open_box"]
    m = vf.vf_mesh_create(v, f)
    t = vf.vf_partition(m, kind, leaf_size=leaf)
    ot = oracle.partition(oracle.mesh(v, f), kind, leaf_size=leaf)
    assert np.array_equal(vf.vf_tree_perm(t), ot.perm)
    nodes = vf.vf_tree_nodes(t)
    assert np.array_equal(nodes["first"], ot.first)
    assert np.array_equal(nodes["count"], ot.count)
    assert np.array_equal(nodes["depth"], ot.depth)
    assert np.array_equal(nodes["parent"], ot.parent)


def test_partition_full_size_dem(vf):
    v, f = synth.fbm_dem_mesh()
    m = vf.vf_mesh_create(v, f)
    t = vf.vf_partition(m, "quad", 64)
    ot = oracle.partition(oracle.mesh(v, f), "quad", 64)
    assert np.array_equal(vf.vf_tree_perm(t), ot.perm)
    assert np.array_equal(vf.vf_tree_nodes(t)["first"], ot.first)


def test_bad_inputs_rejected(vf):
    v, f = synth.tiny_meshes()["facing_pair"]
    bad = f.copy()
    bad[0, 0] = 99
    with pytest.raises(vf.VFError) as e:
        vf.vf_mesh_create(v, bad)
    assert e.value.status == vf.VF_E_INVAL
    with pytest.raises(vf.VFError):
        vf.vf_mesh_create(np.zeros((3, 3)), np.array([[0, 1, 2]]))  # zero extent
