"""Hand-built cell-conversion cases for the oracle (no GPU).

Expected classes are written out by hand from the rules: Sec. 2.2 (interface
cells fill at phi >= 1 + eps and empty at phi <= -eps; gas neighbours of a
filled cell and liquid neighbours of an emptied cell become interface), and
Sec. 2.4 (a cell uncovered by a body becomes gas when its non-obstacle
neighbourhood B(x) holds no liquid, liquid when it holds no gas, interface when
it holds both).
"""
import numpy as np

import oracle
from paper_1201_0351_gb300 import inputs as I

L_, I_, G_, O_ = I.LIQUID, I.INTERFACE, I.GAS, oracle.OBSTACLE

NEIGH = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
         if abs(dx) + abs(dy) + abs(dz) in (1, 2)]


def _layered(n, z_surface, box=None, g=0.0):
    """liquid below z_surface, interface layer (phi 0.5) at z_surface, gas above"""
    flags = np.full((n, n, n), G_, np.uint8)
    fill = np.zeros((n, n, n))
    flags[:z_surface] = L_
    fill[:z_surface] = 1.0
    flags[z_surface] = I_
    fill[z_surface] = 0.5
    rho = np.ones((n, n, n))
    return flags, fill, rho


def _sim(n, flags, fill, rho, boxes=()):
    sc = I.Scenario("conv", n, n, n, 0, 0.7, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 1.0, 1e-2,
                    flags.reshape(-1).copy(), fill.reshape(-1).copy(), rho.reshape(-1).copy(), list(boxes), 0)
    return oracle.OracleSim(sc)


def _ledger_ok(s):
    L = s.ledger()
    return abs(L["M"] - L["M0"] - (L["uncovered"] - L["covered"] - L["lost"] + L["wall"])) <= 1e-12 * L["M0"]


def test_filled_cell_converts_and_gas_neighbours_join_interface():
    n = 8
    flags, fill, rho = _layered(n, 3)
    fill[3, 3, 3] = 1.6
    s = _sim(n, flags, fill, rho)
    s.step(1)
    got = s.fields()["flags"].reshape(n, n, n)
    exp = flags.copy()
    exp[3, 3, 3] = L_
    for dx, dy, dz in NEIGH:
        if dz == 1:
            exp[4 + 0 * dz, 3 + dy, 3 + dx] = I_
    assert np.array_equal(got, exp)
    c = s.counts()
    assert (c["filled"], c["emptied"], c["new_from_gas"], c["new_from_liquid"]) == (1, 0, 5, 0)
    # the five new interface cells each receive the same 1/13 share of the excess
    m = s.fields()["mass"].reshape(n, n, n)
    new = [m[4, 3 + dy, 3 + dx] for dx, dy, dz in NEIGH if dz == 1]
    assert np.ptp(new) == 0.0 and new[0] > 0.03
    # at rest every link's mass exchange vanishes (f = w on both sides), so the
    # filled cell keeps m = 1.6 at rho = 1: its excess e = 0.6 goes in equal
    # shares to its k = 13 interface neighbours after the conversion (the 8 of
    # its own layer and the 5 new ones); other interface cells keep m = 0.5
    e = 1.6 - 1.0
    for dx, dy, dz in NEIGH:
        if dz == 1:
            assert abs(m[4, 3 + dy, 3 + dx] - e / 13) <= 1e-14
        elif dz == 0:
            assert abs(m[3, 3 + dy, 3 + dx] - (0.5 + e / 13)) <= 1e-14
    assert abs(m[3, 0, 0] - 0.5) <= 1e-14 and abs(m[3, 6, 6] - 0.5) <= 1e-14
    assert _ledger_ok(s)


def test_emptied_cell_converts_and_liquid_neighbours_join_interface():
    n = 8
    flags, fill, rho = _layered(n, 3)
    fill[3, 3, 3] = -0.5
    s = _sim(n, flags, fill, rho)
    s.step(1)
    f = s.fields()
    got = f["flags"].reshape(n, n, n)
    exp = flags.copy()
    exp[3, 3, 3] = G_
    for dx, dy, dz in NEIGH:
        if dz == -1:
            exp[2, 3 + dy, 3 + dx] = I_
    assert np.array_equal(got, exp)
    fl = f["fill"].reshape(n, n, n)
    for dx, dy, dz in NEIGH:
        if dz == -1:
            assert 0.9 < fl[2, 3 + dy, 3 + dx] < 1.0  # phi = 1 plus a share of the negative excess
    # at rest the emptied cell keeps m = -0.5 (its excess); the new interface
    # cells start at m = rho = 1, and each of the k = 13 interface neighbours
    # after the conversion (8 of its layer, 5 new) gains e / 13
    m = f["mass"].reshape(n, n, n)
    e = -0.5
    for dx, dy, dz in NEIGH:
        if dz == -1:
            assert abs(m[2, 3 + dy, 3 + dx] - (1.0 + e / 13)) <= 1e-14
        elif dz == 0:
            assert abs(m[3, 3 + dy, 3 + dx] - (0.5 + e / 13)) <= 1e-14
    assert _ledger_ok(s)


def test_emptied_next_to_filled_is_kept():
    n = 8
    flags, fill, rho = _layered(n, 3)
    fill[3, 3, 3] = 1.6
    fill[3, 3, 4] = -0.5
    s = _sim(n, flags, fill, rho)
    s.step(1)
    got = s.fields()["flags"].reshape(n, n, n)
    exp = flags.copy()
    exp[3, 3, 3] = L_
    for dx, dy, dz in NEIGH:
        if dz == 1:
            exp[4, 3 + dy, 3 + dx] = I_
    assert np.array_equal(got, exp)  # (4,3,3) stayed interface, no liquid became interface
    c = s.counts()
    assert (c["filled"], c["emptied"], c["new_from_liquid"]) == (1, 0, 0)
    assert _ledger_ok(s)


def _moving_box_scene(n, z_surface=None):
    if z_surface is None:
        flags = np.full((n, n, n), L_, np.uint8)
        fill = np.ones((n, n, n))
        rho = np.ones((n, n, n))
    else:
        flags, fill, rho = _layered(n, z_surface)
    return flags, fill, rho


def test_box_moving_through_liquid_uncovers_liquid():
    """all-liquid tank: the trailing face becomes liquid, the leading face obstacle"""
    n = 10
    flags, fill, rho = _moving_box_scene(n)
    box = I.Box(center=(4.4999, 5.0, 5.0), half=(2.0, 2.0, 2.0), density_ratio=1e6, vel=(2e-4, 0.0, 0.0),
                mode=I.MODE_FREE)
    s = _sim(n, flags, fill, rho, [box])
    before = s.fields()["flags"].reshape(n, n, n)
    exp0 = flags.copy()
    exp0[3:7, 3:7, 2:6] = O_
    assert np.array_equal(before, exp0)
    s.step(1)
    got = s.fields()["flags"].reshape(n, n, n)
    exp1 = flags.copy()
    exp1[3:7, 3:7, 3:7] = O_
    assert np.array_equal(got, exp1)
    L = s.ledger()
    assert abs(L["covered"] - 16.0) < 1e-2 and abs(L["uncovered"] - 16.0) < 1e-2
    assert _ledger_ok(s)


def test_box_moving_through_surface_uncovers_liquid_interface_gas():
    """box straddling the surface: below the surface an uncovered cell sees no
    gas (-> liquid), at the surface level liquid and gas (-> interface), above
    it no liquid (-> gas)"""
    n = 12
    flags, fill, rho = _moving_box_scene(n, z_surface=6)
    # faces kept off the cell centres: a face through a centre is a tie that
    # the tiny rotation from the surface torque would decide
    box = I.Box(center=(4.4999, 6.0, 6.5), half=(2.0, 2.0, 1.9), density_ratio=1e6, vel=(2e-4, 0.0, 0.0),
                mode=I.MODE_FREE)
    s = _sim(n, flags, fill, rho, [box])
    s.step(1)
    got = s.fields()["flags"].reshape(n, n, n)
    exp = flags.copy()
    exp[5:8, 4:8, 3:7] = O_       # box at its new pose (x cells 3..6, y 4..7, z 5..7)
    exp[5, 4:8, 2] = L_           # uncovered column x = 2
    exp[6, 4:8, 2] = I_
    exp[7, 4:8, 2] = G_
    assert np.array_equal(got, exp)
    fl = s.fields()["fill"].reshape(n, n, n)
    assert np.all(np.abs(fl[6, 4:8, 2] - 0.5) < 0.05)
    assert _ledger_ok(s)


def _pool_with_cell(cell_class, fill_value):
    """A 12^3 closed tank, liquid below z = 4 and an interface layer at z = 4,
    plus one extra cell at (6, 6, 9) of the given class and fill level."""
    n = 12
    flags = np.full((n, n, n), I.GAS, np.uint8)
    fill = np.zeros((n, n, n))
    flags[:4] = I.LIQUID
    fill[:4] = 1.0
    flags[4] = I.INTERFACE
    fill[4] = 0.5
    flags[9, 6, 6] = cell_class
    fill[9, 6, 6] = fill_value
    if cell_class == I.INTERFACE and fill_value > 0.9:
        # an interface cell enclosed by liquid: a liquid blob around it
        flags[8:11, 5:8, 5:8] = I.LIQUID
        fill[8:11, 5:8, 5:8] = 1.0
        flags[9, 6, 6] = I.INTERFACE
        fill[9, 6, 6] = fill_value
        shell = np.zeros_like(flags, dtype=bool)
        shell[7:12, 4:9, 4:9] = True
        shell[8:11, 5:8, 5:8] = False
        flags[shell] = I.INTERFACE
        fill[shell] = 0.5
    return I.Scenario("pool_cell", n, n, n, 0, 0.8, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 1.0, 1e-2,
                      flags.reshape(-1), fill.reshape(-1), np.ones(n ** 3), [], 10)


def _ledger_closes(ref):
    lg = ref.ledger()
    assert abs(lg["M"] - lg["M0"] - (lg["uncovered"] - lg["covered"] - lg["lost"] + lg["wall"])) <= 1e-12 * lg["M0"]


def test_interface_cell_without_liquid_neighbour_empties():
    """A lone interface cell in the gas (a splash with fill 0.3, no liquid
    neighbour) becomes gas at the next step; with no interface neighbour its
    mass leaves through the lost-excess ledger, and the ledger closes."""
    sc = _pool_with_cell(I.INTERFACE, 0.3)
    i = 6 + 12 * (6 + 12 * 9)
    ref = oracle.OracleSim(sc)
    m0 = ref.fields()["mass"][i]
    ref.step(1)
    f = ref.fields()
    assert f["flags"][i] == I.GAS and f["mass"][i] == 0.0
    assert abs(ref.ledger()["lost"] - m0) <= 1e-14
    _ledger_closes(ref)
    assert ref.error == 0


def test_interface_cell_without_gas_neighbour_fills():
    """An interface cell enclosed by liquid (fill 0.95, no gas neighbour)
    becomes liquid at the next step."""
    sc = _pool_with_cell(I.INTERFACE, 0.95)
    i = 6 + 12 * (6 + 12 * 9)
    ref = oracle.OracleSim(sc)
    ref.step(1)
    assert ref.fields()["flags"][i] == I.LIQUID
    _ledger_closes(ref)
    assert ref.error == 0


def test_neighbour_rule_mutation_is_caught():
    oracle.set_mutation(9)
    try:
        ref = oracle.OracleSim(_pool_with_cell(I.INTERFACE, 0.3))
        ref.step(1)
        flag = ref.fields()["flags"][6 + 12 * (6 + 12 * 9)]
    finally:
        oracle.set_mutation(0)
    assert flag == I.INTERFACE


def test_new_interface_cell_takes_the_mean_state_of_its_fluid_neighbours():
    """Sec. 2.2 (reading R8): a gas cell next to a filled cell becomes interface
    with f = f_eq(rho_bar, u_bar), the means over its neighbours that were
    liquid or interface before the conversion (not gas, not the other new
    cells), with each neighbour's velocity that of its last collision,
    u = sum c f / rho - a.  Checked by brute force on a moving surface layer
    with random densities and velocities under gravity, so a wrong neighbour
    set, a velocity without the -a, or a weighted mean all show."""
    n = 8
    rng = np.random.default_rng(11)
    flags, fill, rho = _layered(n, 3)
    fill[3, 3, 3] = 1.6
    rho = 1.0 + 0.02 * (rng.random((n, n, n)) - 0.5)
    vel = 2e-3 * (rng.random((n, n, n, 3)) - 0.5)
    a = np.array([0.0, 0.0, -1e-4])
    sc = I.Scenario("newg", n, n, n, 3, 0.7, tuple(a), (0.0, 0.0, 0.0), 1.0, 1e-2, flags.reshape(-1).copy(),
                    fill.reshape(-1).copy(), rho.reshape(-1).copy(), [], 0, vel=vel.reshape(-1).copy())
    s = oracle.OracleSim(sc)
    s.step(1)
    out = s.fields(want_f=True)
    got = out["flags"].reshape(n, n, n)
    f = out["f"].reshape(19, n, n, n)
    c, w, _ = oracle.lattice()
    new = [(4, 3 + dy, 3 + dx) for dx, dy, dz in NEIGH if dz == 1]
    assert all(got[p] == I_ for p in new)
    for (z, y, x) in new:
        rs, us = [], []
        for dx, dy, dz in NEIGH:
            zz, yy, xx = z + dz, (y + dy) % n, (x + dx) % n
            if not 0 <= zz < n or flags[zz, yy, xx] not in (L_, I_):
                continue
            fk = f[:, zz, yy, xx]
            r = fk.sum()
            rs.append(r)
            us.append((c.T @ fk) / r - a)
        assert len(rs) == 5  # the filled cell and four old interface cells of its layer
        exp = oracle.feq(np.mean(rs), np.mean(us, axis=0))
        assert np.abs(f[:, z, y, x] - exp).max() <= 1e-15
    assert _ledger_ok(s)
