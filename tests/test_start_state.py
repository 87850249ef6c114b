"""Warm-start state preparation (paper Sec. 2.4, Algorithm 1: a new MD run
starts from the final positions and velocities of the database entry most
correlated with it, from the lattice when the database holds none at that
channel height), through mdgp_start_state -- host code, no GPU.  The
snapshot is a liquid from the oracle's MD; removals are checked against the
oracle's Philox4x32-10, insertion energies and the energy bookkeeping
against the oracle's LJ sums."""
import numpy as np
import pytest

from oracle import md as omd

SEED = 20160315
BASE = dict(h=8.0, Lx=10.0, Lz=10.0, density=0.8, T=1.1, g=0.0, steps_eq=0, steps_sample=0, seed=SEED, id=0)


@pytest.fixture(scope="module")
def native():
    from paper_1603_04628_gb300 import build, native as nat
    build.build()
    return nat


@pytest.fixture(scope="module")
def snapshot():
    """A liquid state: 300 oracle steps from the lattice."""
    p = omd.make_params(BASE)
    x, v, a, sp = omd.init(p)
    omd.simulate(p, x, v, a, sp, 0, 300)
    x[:, 0] %= BASE["Lx"]
    x[:, 2] %= BASE["Lz"]
    nf = int((sp == 0).sum())
    assert (sp[:nf] == 0).all() and (sp[nf:] == 1).all()
    xv = np.hstack([x, v]).astype(np.float32)
    return dict(xv=xv, n_fluid=nf, n_wall=len(sp) - nf, h=BASE["h"], Lx=BASE["Lx"], Lz=BASE["Lz"])


def _el(**kw):
    d = dict(BASE)
    d.update(kw)
    return d


def _wrap(d, L):
    return d - L * np.round(d / L)


def _lj_energies(el, xv, n_fluid):
    """Oracle per-atom LJ energies (half of every pair) of a state."""
    p = omd.make_params(el)
    sp = np.zeros(len(xv), np.int32)
    sp[n_fluid:] = 1
    _, _, e = omd.lj_forces(p, np.ascontiguousarray(xv[:, :3], dtype=np.float64), sp, method="brute")
    return e


def test_row_count_matches_the_oracle_geometry(native, snapshot):
    # same element, same reading of App. A: as many fluid and wall atoms as the oracle lays out
    out, kind = native.start_state(_el(id=5), snapshot)
    assert kind == 1
    assert out.shape == (snapshot["n_fluid"] + snapshot["n_wall"], 6)
    # nothing removed or added: the snapshot itself, in double precision
    np.testing.assert_array_equal(out, snapshot["xv"].astype(np.float64))


def test_removal_takes_the_smallest_philox_keys(native, snapshot):
    el = _el(density=0.72, id=9)
    out, kind = native.start_state(el, snapshot)
    assert kind == 1
    nf0, nw = snapshot["n_fluid"], snapshot["n_wall"]
    nf = len(out) - nw
    assert nf < nf0
    keys = [omd.philox4x32_10((i, 0, el["id"], 2), (SEED & 0xFFFFFFFF, SEED >> 32))[0] for i in range(nf0)]
    gone = set(np.argsort(np.array(keys, dtype=np.uint64), kind="stable")[:nf0 - nf].tolist())
    kept = [i for i in range(nf0) if i not in gone]
    src = snapshot["xv"].astype(np.float64)
    np.testing.assert_array_equal(out[:nf], src[kept])
    np.testing.assert_array_equal(out[nf:], src[nf0:])


def test_cold_start_when_the_geometry_differs(native, snapshot):
    # another channel height (the paper's rule), another lateral box, another wall count
    assert native.start_state(_el(h=8.5), snapshot) == (None, 0)
    assert native.start_state(_el(Lx=10.5), snapshot) == (None, 0)
    bad = dict(snapshot, n_wall=snapshot["n_wall"] - 1)
    assert native.start_state(_el(), bad) == (None, 0)


@pytest.mark.parametrize("density", [0.82, 0.86])
def test_insertion_energies_and_bookkeeping(native, snapshot, density):
    el = _el(density=density, id=31)
    out, kind = native.start_state(el, snapshot)
    assert kind == 1
    nf0, nw = snapshot["n_fluid"], snapshot["n_wall"]
    nf = len(out) - nw
    add = nf - nf0
    assert add > 0
    src = snapshot["xv"].astype(np.float64)
    # walls untouched; new atoms inside the slab
    np.testing.assert_array_equal(out[nf:], src[nf0:])
    ins = out[nf0:nf]
    assert (ins[:, 1] >= 0.6).all() and (ins[:, 1] <= el["h"] - 0.6).all()
    # kept atoms: none moved far (only the relaxation of the neighbours of a
    # new atom moves them, at most 0.6 sigma per insertion)
    d = out[:nf0, :3] - src[:nf0, :3]
    d[:, 0] = _wrap(d[:, 0], el["Lx"])
    d[:, 2] = _wrap(d[:, 2], el["Lz"])
    moved = np.linalg.norm(d, axis=1)
    print("inserted %d: kept atoms moved mean %.3f max %.3f, untouched %.2f"
          % (add, moved.mean(), moved.max(), (moved == 0).mean()))
    assert moved.max() < 1.0 and moved.mean() < 0.3
    # the new atoms' oracle LJ energies are moderate (no overlaps)
    e_after = _lj_energies(el, out, nf)
    assert (2.0 * e_after[nf0:nf]).max() < 20.0
    # kept velocities: the snapshot's peculiar velocities scaled by one factor
    vm = src[:nf0, 3:].mean(0)
    a, b = src[:nf0, 3:] - vm, out[:nf0, 3:] - vm
    s = float((a * b).sum() / (a * a).sum())
    np.testing.assert_allclose(b, s * a, rtol=0, atol=1e-12)
    assert 0.5 <= s <= 2.0
    # energy bookkeeping: the kinetic energy removed equals the potential
    # energy added beyond one mean per-atom energy (sum over its pairs) per
    # new atom, both from the oracle's LJ sums
    e_before = _lj_energies(el, np.vstack([src[:nf0], src[nf0:]]), nf0)
    ubar = 2.0 * e_before[:nf0].mean()
    excess = e_after.sum() - e_before.sum() - add * ubar
    kin_after = 0.5 * ((out[:nf, 3:] - vm) ** 2).sum()
    kin_before = kin_after / (s * s)
    assert s * s > 0.25 + 1e-9  # the floor was not reached
    np.testing.assert_allclose(kin_before - kin_after, excess, rtol=1e-8, atol=1e-8)


def test_start_state_is_deterministic(native, snapshot):
    el = _el(density=0.83, id=4)
    a, _ = native.start_state(el, snapshot)
    b, _ = native.start_state(el, snapshot)
    np.testing.assert_array_equal(a, b)
    c, _ = native.start_state(dict(el, id=5), snapshot)
    assert not np.array_equal(a, c)
