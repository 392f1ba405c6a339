"""Slab decomposition of the FSLBM step, exercised on the CPU with the FP64
oracle as the per-rank stepper (gloo, world size 2; no GPU).

The domain is cut along one axis into W slabs.  Each rank holds its slab
plus H ghost layers on both sides and advances it by one oracle step; the
ghost layers are then refilled from the neighbouring ranks' owned layers
(the whole state: post-collision PDFs, cell types, mass, fill level), and
the total mass is summed over ranks in FP64.  A step reads the state within
a fixed radius of a cell: the fill levels of the normals of the fit's block
(two layers), the streamed PDFs, the conversion's neighbourhood; so with H
at least that radius the owned cells equal those of the single-domain step
bit for bit.  H = 3 suffices for the LSQR and TR models and H = 4 for FD (its
K8 smoothing adds a layer); one layer fewer breaks the equality within a
few steps, which the test checks too, so that it would notice a halo that
is too thin.

The ghost layers at the ends of a rank's local array wrap onto each other
inside the oracle and hold wrong values after a step; the exchange replaces
them before they reach an owned cell.  The lost-mass counter of a rank also
counts conversions in its ghost layers and is not compared.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1509_07691_gb300 import synthetic as S  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 6
SHAPE = (24, 24, 24)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _developed(orc, obstacle, curv, seed=3, develop=6):
    """A droplet (or a cap on the floor) in motion with conversions in flight."""
    off = S.centre_offset(seed)
    c = tuple(np.array(SHAPE[::-1]) / 2 - 0.4 + off)
    if obstacle is None:
        phi = orc.fill(orc.geom("sphere", c=c, R=6.3, sub=8), SHAPE)
    else:
        phi = orc.fill(orc.geom("cap", c=(c[0], c[1], 0.5), R=7.3, zw=0.5, sub=8), SHAPE)
    P = orc.params(SHAPE, sigma=5e-4, tau=0.7, theta=np.pi / 3, curv_model=curv)
    st = orc.init_state(P, phi, obstacle)
    fe = np.array([orc.feq(q, 1.0, np.array([0.04, 0.02, -0.03])) for q in range(19)])
    fl = (st.flags & 3) > 0
    st.f[:, fl] = fe[:, None] + S.pdf_noise(seed, SHAPE, 2e-4)[:, fl]
    for _ in range(develop):
        st, _, _, _ = orc.step(P, st)
    return P, st


def _cut(orc, st, axis, lo, hi, n):
    """Layers lo..hi-1 (periodic) of a state along `axis` (0 z, 1 y, 2 x)."""
    idx = np.arange(lo, hi) % n
    return orc.State(np.take(st.f, idx, axis=axis + 1), np.take(st.flags, idx, axis=axis),
                     np.take(st.mass, idx, axis=axis), np.take(st.phi, idx, axis=axis))


def _layers(st, axis, lo, hi):
    """The state's layers lo..hi-1 along `axis`, packed into one FP64 vector."""
    sl = [slice(None)] * 3
    sl[axis] = slice(lo, hi)
    sl = tuple(sl)
    return np.concatenate([st.f[(slice(None),) + sl].ravel(), st.flags[sl].astype(np.float64).ravel(),
                           st.mass[sl].ravel(), st.phi[sl].ravel()])


def _put_layers(st, axis, lo, hi, v):
    sl = [slice(None)] * 3
    sl[axis] = slice(lo, hi)
    sl = tuple(sl)
    nf = st.f[(slice(None),) + sl].size
    nc = st.flags[sl].size
    st.f[(slice(None),) + sl] = v[:nf].reshape(st.f[(slice(None),) + sl].shape)
    st.flags[sl] = v[nf:nf + nc].astype(np.uint8).reshape(st.flags[sl].shape)
    st.mass[sl] = v[nf + nc:nf + 2 * nc].reshape(st.mass[sl].shape)
    st.phi[sl] = v[nf + 2 * nc:].reshape(st.phi[sl].shape)


def _exchange(dist, st, axis, H, n_own, rank, world):
    """Refill the ghost layers from the neighbours' owned layers: every rank
    sends its first and last H owned layers; the lower ghost takes the last
    layers of rank - 1, the upper ghost the first layers of rank + 1."""
    first = torch.from_numpy(_layers(st, axis, H, 2 * H))
    last = torch.from_numpy(_layers(st, axis, n_own, n_own + H))
    mine = torch.cat([first, last])
    got = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(got, mine)
    k = first.numel()
    _put_layers(st, axis, 0, H, got[(rank - 1) % world][k:].numpy())
    _put_layers(st, axis, n_own + H, n_own + 2 * H, got[(rank + 1) % world][:k].numpy())


def _rank_main(rank, world, port, cases, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import oracle as orc

    dist.init_process_group("gloo", rank=rank, world_size=world)
    results = []
    try:
        for name, walls, curv, axis, H in cases:
            obstacle = S.obstacle_mask(SHAPE, (0, SHAPE[0] - 1)) if walls else None
            P, ref = _developed(orc, obstacle, curv)
            n = SHAPE[axis]
            lo, hi = rank * n // world, (rank + 1) * n // world
            n_own = hi - lo
            shape = list(SHAPE)
            shape[axis] = n_own + 2 * H
            Pl = orc.params(tuple(shape), sigma=P.sigma, tau=P.tau, theta=P.theta, curv_model=P.curv_model)
            loc = _cut(orc, ref, axis, lo - H, hi + H, n)
            own = [slice(None)] * 3
            own[axis] = slice(H, H + n_own)
            own = tuple(own)
            Po = orc.params(tuple(shape[:axis] + [n_own] + shape[axis + 1:]), sigma=P.sigma, tau=P.tau,
                            theta=P.theta, curv_model=P.curv_model)
            equal_steps, conversions, mass_err = 0, 0, 0.0
            for _ in range(STEPS):
                ref, counts, _, _ = orc.step(P, ref)
                conversions += int(counts[3] + counts[4] + counts[5] + counts[6])
                loc, _, _, _ = orc.step(Pl, loc)
                mine = _cut(orc, ref, axis, lo, hi, n)
                same = (np.array_equal(loc.flags[own], mine.flags) and np.array_equal(loc.mass[own], mine.mass)
                        and np.array_equal(loc.phi[own], mine.phi)
                        and np.array_equal(loc.f[(slice(None),) + own], mine.f))
                flag = torch.tensor([1 if same else 0])
                dist.all_reduce(flag, op=dist.ReduceOp.MIN)
                if flag.item() == 0:
                    break
                equal_steps += 1
                # total mass over the ranks' owned cells, FP64 sum
                ms = orc.State(loc.f[(slice(None),) + own].copy(), loc.flags[own].copy(), loc.mass[own].copy(),
                               loc.phi[own].copy())
                m = torch.tensor([orc.mass(Po, ms)], dtype=torch.float64)
                dist.all_reduce(m)
                mass_err = max(mass_err, abs(m.item() - orc.mass(P, ref)) / orc.mass(P, ref))
                _exchange(dist, loc, axis, H, n_own, rank, world)
            results.append((name, equal_steps, conversions, mass_err))
    finally:
        dist.destroy_process_group()
    if rank == 0:
        with open(out, "w") as fh:
            json.dump(results, fh)


def _run(cases, out, world=2):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, cases, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
        assert p.exitcode == 0
    with open(out) as fh:
        return json.load(fh)


@pytest.mark.slow
def test_slab_decomposition_reproduces_the_step(orc, tmp_path):
    # (name, obstacle walls, curvature model, cut axis, ghost layers)
    cases = [("droplet LSQR z", False, 0, 0, 3), ("cap at walls LSQR y", True, 0, 1, 3),
             ("droplet FD z", False, 1, 0, 4), ("cap at walls FD y", True, 1, 1, 4),
             ("droplet TR z", False, 2, 0, 3),
             ("droplet LSQR z, halo too thin", False, 0, 0, 2), ("droplet FD z, halo too thin", False, 1, 0, 3)]
    res = {name: (eq, conv, merr) for name, eq, conv, merr in _run(cases, str(tmp_path / "slabs.json"))}
    for name, _, _, _, _ in cases:
        eq, conv, merr = res[name]
        if "too thin" in name:
            assert eq < STEPS, f"{name}: a halo one layer thinner should break the equality"
        else:
            assert eq == STEPS, f"{name}: owned cells differ from the single-domain step after {eq} steps"
            assert conv > 20, f"{name}: the case must convert cells across the cut"
            assert merr < 1e-12, f"{name}: FP64 mass sum over the ranks off by {merr}"


@pytest.mark.slow
def test_three_slabs(orc, tmp_path):
    """Three ranks: the lower and upper neighbours of a rank differ."""
    cases = [("droplet LSQR z, 3 ranks", False, 0, 0, 3), ("cap at walls FD y, 3 ranks", True, 1, 1, 4)]
    res = _run(cases, str(tmp_path / "slabs3.json"), world=3)
    for name, eq, conv, merr in res:
        assert eq == STEPS and conv > 20 and merr < 1e-12, (name, eq, conv, merr)

