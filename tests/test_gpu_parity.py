"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Element-by-element comparisons on seeded inputs at sizes the oracle runs in
seconds (several 128-node tiles plus a ragged tail), every wetting scheme,
both kernel schedules, every storage format, and the edge cases of the
method. Tolerances: FP64 storage 1e-11 (rounding order only); FP32 storage
max|drho|/rho <= 1e-5 and max|du| <= 1e-7 after 1000 steps.
"""
import hashlib

import numpy as np
import pytest

import oracle
from paper_2009_12584_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2009_12584_gb300 import lbm  # noqa: E402

KERNELS = ["two_pass", "fused", "tiled", "halo", "tma"]

WETTINGS = {
    "mc": (dict(bc=oracle.BC_MARTYS_CHEN, G_s=(-0.2, 0.2)), ("martys_chen", dict(G_s=(-0.2, 0.2)))),
    "llkc": (dict(bc=oracle.BC_LLKC, G_s=(-0.5, 0.5)), ("llkc", dict(G_s=(-0.5, 0.5)))),
    "llkc_self": (dict(bc=oracle.BC_LLKC, G_s=(-0.5, 0.3), pairing=oracle.PAIR_SELF),
                  ("llkc", dict(G_s=(-0.5, 0.3), pairing=lbm.PAIR_SELF))),
    "improved": (dict(bc=oracle.BC_VIRTUAL_AVG, G_s=(3.0, 3.0), chi=(1.2, 0.8)),
                 ("virtual_avg", dict(G_s=(3.0, 3.0), chi=(1.2, 0.8)))),
    "improved_self_d2q9": (dict(bc=oracle.BC_VIRTUAL_AVG, G_s=(2.5, 3.5), chi=(0.9, 1.3),
                                pairing=oracle.PAIR_SELF, avg_stencil=9),
                           ("virtual_avg", dict(G_s=(2.5, 3.5), chi=(0.9, 1.3), pairing=lbm.PAIR_SELF,
                                                avg_stencil=9))),
    "constant": (dict(bc=oracle.BC_CONSTANT, G_s=(3.0, 3.0), rho_s=(0.3, 0.7)),
                 ("constant", dict(G_s=(3.0, 3.0), rho_s=(0.3, 0.7)))),
}


_ORACLE_CACHE = {}


def _oracle_run(nx, ny, mask, rA, rB, steps, wet, periodic, tau, ux, uy):
    """Oracle state after ``steps``; cached so that both kernel schedules are
    compared with one oracle run."""
    h = hashlib.sha1()
    for a in (mask, rA, rB, ux, uy):
        h.update(b"none" if a is None else np.ascontiguousarray(a).tobytes())
    key = (nx, ny, steps, wet, periodic, tau, h.hexdigest())
    if key not in _ORACLE_CACHE:
        okw, _ = WETTINGS[wet]
        o = oracle.Oracle(nx, ny, mask, tau=tau, periodic_x=periodic[0], periodic_y=periodic[1], **okw)
        o.init(rA, rB, ux, uy).step(steps)
        _ORACLE_CACHE[key] = o
    return _ORACLE_CACHE[key]


def run_pair(nx, ny, mask, rA, rB, steps, wet, *, periodic=(False, False), storage="fp64",
             kernel="two_pass", tau=(1.0, 1.0), ux=None, uy=None):
    _, (kind, gkw) = WETTINGS[wet]
    o = _oracle_run(nx, ny, mask, rA, rB, steps, wet, tuple(periodic), tuple(tau), ux, uy)
    sim = lbm.Simulation(nx, ny, tau=tau, periodic_x=periodic[0], periodic_y=periodic[1],
                         storage=storage, kernel=kernel)
    sim.set_geometry(mask).set_wetting(kind, **gkw).init_fields(rA, rB, ux, uy).step(steps)
    rhoA, rhoB, u = sim.moments()
    torch.cuda.synchronize()
    return o, sim, (rhoA.cpu().numpy(), rhoB.cpu().numpy(), u.cpu().numpy())


def errors(o, gpu, mask):
    rho, rt, F, u = o.fields()
    fl = mask == 0
    d_rho = max((np.abs(gpu[0] - rho[0])[fl] / rho[0][fl]).max(), (np.abs(gpu[1] - rho[1])[fl] / rho[1][fl]).max())
    d_u = np.abs(gpu[2] - u)[:, fl].max()
    return d_rho, d_u


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("wet", list(WETTINGS))
def test_fp64_inclined_wall(wet, kernel):
    """FP64 storage: agreement to rounding on an off-grid wall (two 128-node
    tiles plus a ragged tail), every wetting scheme."""
    nx, ny = 150, 70
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, 12)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 12)
    o, sim, g = run_pair(nx, ny, mask, rA, rB, 200, wet, kernel=kernel)
    d_rho, d_u = errors(o, g, mask)
    assert d_rho < 1e-11 and d_u < 1e-12, (d_rho, d_u)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("wet", ["mc", "llkc", "improved"])
def test_fp64_periodic_salt(wet, kernel):
    """Fully periodic box with isolated solid nodes, one-node gaps and
    corners; random densities and velocities exercise every term."""
    nx, ny = 37, 29
    mask = inputs.random_solid_mask(nx, ny, seed=11, fraction=0.15)
    rA, rB, ux, uy = inputs.random_fields(nx, ny, seed=12, lo=0.2, hi=0.8, umax=0.02)
    o, sim, g = run_pair(nx, ny, mask, rA, rB, 60, wet, periodic=(True, True), kernel=kernel,
                         tau=(0.8, 1.3), ux=ux, uy=uy)
    d_rho, d_u = errors(o, g, mask)
    assert d_rho < 1e-11 and d_u < 1e-12, (d_rho, d_u)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("wet", ["mc", "llkc", "improved"])
def test_fp32_inclined_wall_1000_steps(wet, kernel):
    """FP32 storage and arithmetic after 1000 steps: max|drho|/rho <= 1e-5,
    max|du| <= 1e-7 against FP64."""
    nx, ny = 200, 100
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, 15)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 15)
    o, sim, g = run_pair(nx, ny, mask, rA, rB, 1000, wet, storage="fp32", kernel=kernel)
    d_rho, d_u = errors(o, g, mask)
    assert d_rho <= 1e-5 and d_u <= 1e-7, (d_rho, d_u)


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp32_flat_wall_droplet_at_rest(kernel):
    """100x50 channel periodic in x, flat wall along y = 0, semicircular
    droplet (1.0 in, 0.03 out), Martys-Chen at neutral wetting: parity after
    1000 steps and no sliding."""
    nx, ny = 100, 50
    mask = inputs.flat_wall_mask(nx, ny)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, 0.5, 15, 1.0, 0.03)
    okw = dict(bc=oracle.BC_MARTYS_CHEN, G_s=(0.0, 0.0))
    o = oracle.Oracle(nx, ny, mask, periodic_x=True, **okw).init(rA, rB).step(1000)
    sim = lbm.Simulation(nx, ny, periodic_x=True, storage="fp32", kernel=kernel)
    sim.set_geometry(mask).set_wetting("martys_chen", G_s=(0.0, 0.0)).init_fields(rA, rB).step(1000)
    rhoA, rhoB, u = sim.moments()
    g = (rhoA.cpu().numpy(), rhoB.cpu().numpy(), u.cpu().numpy())
    d_rho, d_u = errors(o, g, mask)
    assert d_rho <= 1e-5 and d_u <= 1e-7, (d_rho, d_u)
    w = np.maximum(g[0] - 0.03, 0)
    assert abs((w * g[2][0]).sum() / w.sum()) < 1e-7


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("nx,ny,per", [(4, 4, (True, True)), (5, 4, (True, False)), (131, 9, (True, True)),
                                       (129, 6, (False, True)), (8, 130, (True, False))])
def test_fp64_edge_sizes(nx, ny, per, kernel):
    """Smallest grids, odd and ragged sizes, periodic axes shorter than two
    ghost layers."""
    mask = inputs.random_solid_mask(nx, ny, seed=nx * 1000 + ny, fraction=0.1, periodic_x=per[0],
                                    periodic_y=per[1])
    rA, rB, ux, uy = inputs.random_fields(nx, ny, seed=3, lo=0.2, hi=0.9, umax=0.01)
    o, sim, g = run_pair(nx, ny, mask, rA, rB, 25, "improved", periodic=per, kernel=kernel, ux=ux, uy=uy)
    d_rho, d_u = errors(o, g, mask)
    assert d_rho < 1e-11 and d_u < 1e-12, (d_rho, d_u)


@pytest.mark.parametrize("kernel", KERNELS)
def test_fp64_no_solid_and_isolated_fluid(kernel):
    """A box with no solid node, and one whose only fluid node has eight
    solid neighbours (everything bounces back)."""
    nx, ny = 16, 12
    rA, rB, ux, uy = inputs.random_fields(nx, ny, seed=4, lo=0.2, hi=0.9, umax=0.02)
    mask = np.zeros((ny, nx), np.uint8)
    o, sim, g = run_pair(nx, ny, mask, rA, rB, 30, "mc", periodic=(True, True), kernel=kernel, ux=ux, uy=uy)
    assert max(errors(o, g, mask)) < 1e-11
    mask = np.ones((ny, nx), np.uint8)
    mask[5, 7] = 0
    o, sim, g = run_pair(nx, ny, mask, rA, rB, 30, "improved", kernel=kernel, ux=ux, uy=uy)
    assert max(errors(o, g, mask)) < 1e-11


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_auto_schedule_follows_wetting_scheme(storage):
    """AUTO runs the halo schedule under the one-node-reach schemes and the
    tiled one under the improved scheme; switching the scheme mid-run (halo
    -> tiled -> halo, the density plane recomputed where needed) gives the
    two-pass schedule's results bit for bit."""
    nx, ny = 70, 45
    mask = inputs.random_solid_mask(nx, ny, seed=21, fraction=0.15, periodic_x=True, periodic_y=True)
    rA, rB, ux, uy = inputs.random_fields(nx, ny, seed=22, lo=0.2, hi=0.9, umax=0.01)
    plan = [("mc", 9), ("improved", 7), ("llkc", 6), ("constant", 5), ("improved", 4)]
    out = {}
    for kernel in ("auto", "two_pass"):
        sim = lbm.Simulation(nx, ny, periodic_x=True, periodic_y=True, storage=storage, kernel=kernel)
        sim.set_geometry(mask)
        for j, (wet, steps) in enumerate(plan):
            kind, gkw = WETTINGS[wet][1]
            sim.set_wetting(kind, **gkw)
            if j == 0:
                sim.init_fields(rA, rB, ux, uy)
            sim.step(steps)
        out[kernel] = [t.cpu() for t in sim.moments()] + [np.asarray(sim.mass())]
        sim.close()
    for a, b in zip(out["auto"][:3], out["two_pass"][:3]):
        assert torch.equal(a, b)
    assert np.array_equal(out["auto"][3], out["two_pass"][3])


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("kernel", KERNELS)
def test_no_fluid_node(kernel, storage):
    """An all-solid box, walled and periodic: every schedule runs over empty
    lists, tiles and work lists, and the state stays what the oracle keeps
    (no mass, zero densities and velocities, no interface-solid cell)."""
    nx, ny = 40, 20
    mask = np.ones((ny, nx), np.uint8)
    rA, rB, ux, uy = inputs.random_fields(nx, ny, seed=6, lo=0.2, hi=0.9, umax=0.01)
    for periodic in ((False, False), (True, True)):
        o, sim, g = run_pair(nx, ny, mask, rA, rB, 5, "improved", periodic=periodic, storage=storage,
                             kernel=kernel)
        rho, _, _, u = o.fields()
        assert sim.interface_count() == 0
        assert list(sim.mass()) == [0.0, 0.0] and list(o.mass()) == [0.0, 0.0]
        for a, b in ((g[0], rho[0]), (g[1], rho[1]), (g[2], u)):
            assert np.array_equal(a, b)
        sim.close()


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_forces_and_populations_api(storage):
    nx, ny = 60, 40
    mask = inputs.inclined_wall_mask(nx, ny, 30.0, 8)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 8)
    o, sim, g = run_pair(nx, ny, mask, rA, rB, 17, "improved", storage=storage)
    rho, rt, F, u = o.fields()
    tol = 1e-12 if storage == "fp64" else 2e-6
    np.testing.assert_allclose(sim.forces().cpu().numpy(), F, rtol=0, atol=tol)
    np.testing.assert_allclose(sim.populations().cpu().numpy(), o.f, rtol=0, atol=tol)
    m = sim.mass()
    np.testing.assert_allclose(m, o.mass(), rtol=1e-13 if storage == "fp64" else 1e-6)


def test_checkpoint_restore_is_exact():
    nx, ny = 70, 50
    mask = inputs.inclined_wall_mask(nx, ny, 10.0, 9)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 9)
    a = lbm.Simulation(nx, ny, storage="fp64")
    a.set_geometry(mask).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=(1.1, 0.9)).init_fields(rA, rB).step(30)
    f = a.populations().clone()
    a.step(20)
    b = lbm.Simulation(nx, ny, storage="fp64")
    b.set_geometry(mask).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=(1.1, 0.9)).set_populations(f).step(20)
    assert torch.equal(a.populations(), b.populations())


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
@pytest.mark.parametrize("wet", ["mc", "llkc_self", "improved", "improved_self_d2q9", "constant"])
@pytest.mark.parametrize("case", ["porous_periodic", "wall_walled"])
def test_single_pass_matches_two_pass_bitwise(storage, wet, case):
    """The schedules run the same node arithmetic and the same density sums
    in the same order, so they must agree bit for bit (several 30-column
    strips of the marching kernel plus a ragged one, row segments; several
    32 x 14 tiles of the tiled kernel plus ragged ones in x and y)."""
    if case == "porous_periodic":
        nx, ny, per = 157, 131, (True, True)
        mask = inputs.porous_disks(nx, ny, 0.35, rmin=3, rmax=9, seed=5)
        rA, rB = inputs.pore_droplets(mask, 0.3, rmin=3, rmax=8, seed=6)
    else:
        nx, ny, per = 123, 77, (False, False)
        mask = inputs.inclined_wall_mask(nx, ny, 20.0, 12)
        rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 12)
    _, (kind, gkw) = WETTINGS[wet]
    outs = []
    for kernel in KERNELS:
        s = lbm.Simulation(nx, ny, periodic_x=per[0], periodic_y=per[1], storage=storage, kernel=kernel)
        s.set_geometry(mask).set_wetting(kind, **gkw).init_fields(rA, rB).step(37)
        outs.append((s.populations(), s.moments(), s.mass()))
    for other in outs[1:]:
        assert torch.equal(outs[0][0], other[0])
        for a, b in zip(outs[0][1], other[1]):
            assert torch.equal(a, b)
        assert np.array_equal(outs[0][2], other[2])


@pytest.mark.parametrize("kernel", KERNELS)
def test_deterministic(kernel):
    nx, ny = 150, 64
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, 10)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 10)
    outs = []
    for _ in range(2):
        s = lbm.Simulation(nx, ny, storage="fp32", kernel=kernel)
        s.set_geometry(mask).set_wetting("improved", G_s=(3.0, 3.0), chi=(1.2, 0.8)).init_fields(rA, rB).step(50)
        outs.append((s.populations(), s.mass()))
    assert torch.equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_interface_count_matches_oracle():
    nx, ny = 120, 90
    mask = inputs.circle_surface_mask(nx, ny, 60, 20, 30)
    sim = lbm.Simulation(nx, ny, periodic_x=True, periodic_y=True)
    sim.set_geometry(mask)
    o = oracle.Oracle(nx, ny, mask, periodic_x=True, periodic_y=True)
    assert sim.interface_count() == int(o.interface_solid().sum())


def test_run_host_matches_device_path():
    nx, ny = 90, 60
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, 10)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 10)
    a = lbm.Simulation(nx, ny)
    a.set_geometry(mask).set_wetting("llkc", G_s=(-0.5, 0.5)).init_fields(rA, rB).step(40)
    rhoA, rhoB, u = a.moments()
    b = lbm.Simulation(nx, ny)
    outs = [np.zeros((ny, nx)) for _ in range(4)]
    b.run_host(lbm.make_wetting("llkc", G_s=(-0.5, 0.5)), mask.copy(), rA.copy(), rB.copy(), 40, outs)
    assert np.array_equal(outs[0], rhoA.cpu().numpy())
    assert np.array_equal(outs[2], u[0].cpu().numpy())


def test_run_host_f32_matches_device_path():
    """The FP32 host interface starts from the FP32-rounded densities and
    returns the FP32-rounded moments of the same run (FP32 storage computes
    in FP32, so the rounding of the outputs is exact)."""
    nx, ny = 90, 60
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, 10)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 10)
    rA32, rB32 = rA.astype(np.float32), rB.astype(np.float32)
    a = lbm.Simulation(nx, ny)
    a.set_geometry(mask).set_wetting("llkc", G_s=(-0.5, 0.5))
    a.init_fields(rA32.astype(np.float64), rB32.astype(np.float64)).step(40)
    rhoA, rhoB, u = a.moments()
    b = lbm.Simulation(nx, ny)
    outs = [np.zeros((ny, nx), np.float32) for _ in range(4)]
    b.run_host_f32(lbm.make_wetting("llkc", G_s=(-0.5, 0.5)), mask.copy(), rA32, rB32, 40, outs)
    assert np.array_equal(outs[0], rhoA.cpu().numpy().astype(np.float32))
    assert np.array_equal(outs[1], rhoB.cpu().numpy().astype(np.float32))
    assert np.array_equal(outs[2], u[0].cpu().numpy().astype(np.float32))
    assert np.array_equal(outs[3], u[1].cpu().numpy().astype(np.float32))


def test_errors_are_status_codes():
    nx, ny = 16, 16
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(nx, ny, tau=(0.5, 1.0))
    assert e.value.status == lbm.ERR_ARG
    sim = lbm.Simulation(nx, ny)
    with pytest.raises(lbm.LbmError) as e:
        sim.step(1)
    assert e.value.status == lbm.ERR_STATE
    with pytest.raises(lbm.LbmError) as e:
        sim.set_geometry(np.zeros((ny, nx), np.uint8))  # fluid on walled borders
    assert e.value.status == lbm.ERR_ARG
    with pytest.raises(lbm.LbmError) as e:
        sim.set_wetting("virtual_avg", chi=(0.0, 1.0))
    assert e.value.status == lbm.ERR_ARG
    small = lbm.Simulation(nx, ny, max_interface=3)
    with pytest.raises(lbm.LbmError) as e:
        small.set_geometry(inputs.border_walls(nx, ny))
    assert e.value.status == lbm.ERR_SPACE


@pytest.mark.parametrize("vref", [False, True], ids=["rho_refs", "velocity_refs"])
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_reduced_storage_checkpoint_roundtrip(storage, vref):
    """Populations written back through lbm_set_populations are re-encoded
    relative to each node's own density and read back to the precision of
    the format."""
    nx, ny = 40, 30
    mask = inputs.random_solid_mask(nx, ny, seed=5, fraction=0.1)
    rA, rB, ux, uy = inputs.random_fields(nx, ny, seed=6, lo=0.2, hi=0.9, umax=0.02)
    a = lbm.Simulation(nx, ny, periodic_x=True, periodic_y=True, storage="fp64")
    a.set_geometry(mask).set_wetting("llkc", G_s=(-0.5, 0.5)).init_fields(rA, rB, ux, uy).step(5)
    f = a.populations()
    b = lbm.Simulation(nx, ny, periodic_x=True, periodic_y=True, storage=storage, velocity_refs=vref)
    b.set_geometry(mask).set_wetting("llkc", G_s=(-0.5, 0.5)).set_populations(f)
    eps = 2.0 ** -11 if storage == "fp16" else 2.0 ** -8
    # deviations are a few percent of f at most here
    err = (b.populations() - f).abs().max().item()
    assert err <= 0.1 * eps, err


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batch_matches_individual_runs(storage):
    """Simulations advanced together by one batch end bit-identical to the
    same simulations advanced one by one (same kernels, same arithmetic)."""
    work = inputs.batched_workload(7, seed=3, size_scale=0.3)
    def make():
        sims = []
        for w in work:
            s = lbm.Simulation(w["nx"], w["ny"], storage=storage)
            s.set_geometry(w["mask"]).set_wetting(w["bc"], **w["wetting"]).init_fields(w["rhoA"], w["rhoB"])
            sims.append(s)
        return sims
    solo = make()
    for s in solo:
        s.step(37)
    group = make()
    b = lbm.Batch(group)
    b.step(5)             # direct launches
    b.set_graph_steps(8)
    b.step(32)            # four graph replays
    for a, c in zip(solo, group):
        assert torch.equal(a.populations(), c.populations())
    assert b.launch_count > 0


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_batch_tiled_schedule_matches_individual_runs(storage):
    """The batched tiled schedule (one Eq. 8 launch and one tiled launch over
    all members' tiles per step) leaves every member bit-identical to the
    same simulation stepped alone, with direct launches and graph replays."""
    work = inputs.batched_workload(7, seed=3, size_scale=0.3)
    def make():
        sims = []
        for w in work:
            s = lbm.Simulation(w["nx"], w["ny"], storage=storage)
            s.set_geometry(w["mask"]).set_wetting(w["bc"], **w["wetting"]).init_fields(w["rhoA"], w["rhoB"])
            sims.append(s)
        return sims
    solo = make()
    for s in solo:
        s.step(41)
    group = make()
    b = lbm.Batch(group).set_schedule("tiled")
    assert b.config()[0] == "tiled"
    b.step(5)             # direct launches
    b.set_graph_steps(8)
    b.step(32)            # four graph replays
    b.set_schedule("two_pass")
    b.step(4)             # switching schedules keeps the state
    for a, c in zip(solo, group):
        assert torch.equal(a.populations(), c.populations())
        assert np.array_equal(a.mass(), c.mass())


@pytest.mark.parametrize("schedule", ["two_pass", "tiled"])
def test_batch_members_match_oracle(schedule):
    """Members of one batch (different sizes, wall angles and wetting
    schemes) compared directly with their own oracle runs: FP64 storage
    within rounding order (1e-11 relative density, 1e-12 velocity)."""
    work = inputs.batched_workload(5, seed=21, size_scale=0.2)
    sims = []
    for w in work:
        s = lbm.Simulation(w["nx"], w["ny"], storage="fp64")
        s.set_geometry(w["mask"]).set_wetting(w["bc"], **w["wetting"]).init_fields(w["rhoA"], w["rhoB"])
        sims.append(s)
    b = lbm.Batch(sims).set_schedule(schedule)
    b.set_graph_steps(8)
    b.step(60)
    bcs = {"martys_chen": oracle.BC_MARTYS_CHEN, "llkc": oracle.BC_LLKC, "virtual_avg": oracle.BC_VIRTUAL_AVG}
    assert len({w["bc"] for w in work}) >= 2
    for i in (0, 2, 4):
        w = work[i]
        o = oracle.Oracle(w["nx"], w["ny"], w["mask"], bc=bcs[w["bc"]], **w["wetting"]).init(w["rhoA"], w["rhoB"])
        o.step(60)
        rA, rB, u = (v.cpu().numpy() for v in sims[i].moments())
        rho_o, _, _, u_o = o.fields()
        fl = w["mask"] == 0
        assert np.abs(rA - rho_o[0])[fl].max() / rho_o[0][fl].min() < 1e-11, i
        assert np.abs(rB - rho_o[1])[fl].max() / rho_o[1][fl].min() < 1e-11, i
        assert np.abs(u - u_o)[:, fl].max() < 1e-12, i


def test_batch_autotune_and_members_stay_usable():
    work = inputs.batched_workload(5, seed=4, size_scale=0.25)
    sims = []
    for w in work:
        s = lbm.Simulation(w["nx"], w["ny"])
        s.set_geometry(w["mask"]).set_wetting(w["bc"], **w["wetting"]).init_fields(w["rhoA"], w["rhoB"])
        sims.append(s)
    m0 = [s.mass() for s in sims]
    b = lbm.Batch(sims)
    threads, steps = b.autotune(8)
    assert threads in (128, 256) and steps in (2, 8, 32)
    assert b.config()[0] in ("two_pass", "tiled") and b.config()[2] == steps
    b.step(10)
    for s, m in zip(sims, m0):
        np.testing.assert_allclose(s.mass(), m, rtol=1e-5)
        s.step(1)  # members can still be stepped alone


def test_l2_fetch_granularity_hint_changes_no_result():
    nx, ny = 96, 64
    mask = inputs.inclined_wall_mask(nx, ny, 20.0, 10)
    rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 10)
    outs = []
    prev = lbm.set_l2_fetch_granularity(128)
    try:
        for g in (128, 32):
            assert lbm.set_l2_fetch_granularity(g) in (32, 64, 128)
            s = lbm.Simulation(nx, ny, storage="fp32")
            s.set_geometry(mask).set_wetting("virtual_avg", G_s=(3.0, 3.0), chi=(1.2, 0.8)).init_fields(rA, rB)
            outs.append(s.step(30).populations())
        assert torch.equal(outs[0], outs[1])
        with pytest.raises(lbm.LbmError):
            lbm.set_l2_fetch_granularity(48)
        assert lbm.set_l2_fetch_granularity(prev) == 32
    finally:
        lbm.set_l2_fetch_granularity(prev)


@pytest.mark.parametrize("kernel", KERNELS)
def test_geometry_change_rebuilds_lists(kernel):
    """A context whose geometry is replaced continues exactly like a fresh
    context on the new geometry (flags, fluid, interface and tile lists are
    rebuilt; the density planes are cleared)."""
    nx, ny = 97, 41
    m1 = inputs.porous_disks(nx, ny, 0.3, rmin=3, rmax=7, seed=11)
    m2 = inputs.porous_disks(nx, ny, 0.45, rmin=2, rmax=6, seed=12)
    r1 = inputs.pore_droplets(m1, 0.3, rmin=3, rmax=6, seed=13)
    r2 = inputs.pore_droplets(m2, 0.3, rmin=3, rmax=6, seed=14)
    wet = dict(G_s=(3.0, 3.0), chi=(1.2, 0.8))
    a = lbm.Simulation(nx, ny, periodic_x=True, periodic_y=True, storage="fp32", kernel=kernel)
    a.set_geometry(m1).set_wetting("virtual_avg", **wet).init_fields(*r1).step(15)
    a.set_geometry(m2).init_fields(*r2).step(20)
    b = lbm.Simulation(nx, ny, periodic_x=True, periodic_y=True, storage="fp32", kernel=kernel)
    b.set_geometry(m2).set_wetting("virtual_avg", **wet).init_fields(*r2).step(20)
    assert a.interface_count() == b.interface_count()
    assert torch.equal(a.populations(), b.populations())
    assert np.array_equal(a.mass(), b.mass())


@pytest.mark.parametrize("vref", [False, True], ids=["rho_refs", "velocity_refs"])
@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("wet", ["mc", "improved", "improved_self_d2q9"])
@pytest.mark.parametrize("case", ["porous_periodic", "wall_walled"])
def test_tiled_16bit_matches_two_pass_bitwise(storage, wet, case, vref):
    """With 16-bit storage the tiled kernel decodes with the writers'
    densities of the step before, encodes with its own, and sums the values
    the next step decodes: the same bits as the two-pass schedule. The tiled
    run is interrupted by a moments() call, after which its densities are
    computed again."""
    if case == "porous_periodic":
        nx, ny, per = 157, 131, (True, True)
        mask = inputs.porous_disks(nx, ny, 0.35, rmin=3, rmax=9, seed=5)
        rA, rB = inputs.pore_droplets(mask, 0.3, rmin=3, rmax=8, seed=6)
    else:
        nx, ny, per = 123, 77, (False, False)
        mask = inputs.inclined_wall_mask(nx, ny, 20.0, 12)
        rA, rB = inputs.sharp_droplet(nx, ny, nx / 2, ny / 2, 12)
    _, (kind, gkw) = WETTINGS[wet]
    outs = []
    for kernel in ("two_pass", "tiled"):
        s = lbm.Simulation(nx, ny, periodic_x=per[0], periodic_y=per[1], storage=storage, kernel=kernel,
                           velocity_refs=vref)
        s.set_geometry(mask).set_wetting(kind, **gkw).init_fields(rA, rB).step(13)
        s.moments()
        s.step(24)
        outs.append((s.populations(), s.moments(), s.mass()))
    assert torch.equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][1]):
        assert torch.equal(a, b)
    assert np.array_equal(outs[0][2], outs[1][2])
