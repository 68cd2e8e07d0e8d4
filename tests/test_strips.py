"""Row-strip decomposition (one image over several ranks) on CPU.

The driver in ``paper_1409_7474_gb300.strips`` owns the partition, the
(r + 1)-row halo exchange of the LSF and the per-iteration all-reduce of
(|P|, sign changes, sum_P I_b); the arithmetic of a strip is a callback.  Here
the callback is the FP64 oracle (``_strip_oracle.OracleCompute``), and the
ranks are gloo processes: every rank's owned rows must be those of the
oracle's whole-image evolution, for the region term with one and three
bands, the edge term, re-initialisation every iteration (one-byte sign
halos) and every third iteration (float halos), and an early stop.  A driver
whose halo exchange does nothing must fail the same comparison.
"""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from _strip_oracle import OracleCompute
from paper_1409_7474_gb300 import scenes, strips

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (H, W, B, term, ts, iterations, reinit_period, early_stop_frac)
CASES = [
    (37, 29, 1, "region", 9, 12, 1, 0.0),
    (41, 30, 3, "region", 7, 10, 3, 0.0),
    (39, 26, 1, "edge", 9, 10, 1, 0.0),
    (46, 33, 1, "region", 5, 80, 1, 0.0435),
]


def case_inputs(H, W, B, term, ts):
    """A seeded two-level scene (B bands: the rectangle with band-dependent
    contrast), an off-centre circle as phi0, and g for the edge term."""
    img, _, _ = scenes.rect_scene(H, W, W // 2, H // 3, noise=0.08, seed_pos=H,
                                  seed_noise=W)
    img = np.concatenate([img * (1.0 - 0.2 * b) + 0.1 * b for b in range(B)]).astype(np.float64)
    phi0 = scenes.circle_phi(H, W, cy=H * 0.45, cx=W * 0.55, radius=min(H, W) / 3.5)
    phi0 = phi0.astype(np.float64)
    if term == "edge":
        phi0 = scenes.box_phi(H, W, [(2, 2, H - 2, W - 2)]).astype(np.float64)
    g = oracle.edge_indicator(img, 1.0, 5, 255.0) if term == "edge" else None
    return img, phi0, g


def whole_image(case):
    H, W, B, term, ts, iters, period, frac = case
    img, phi0, g = case_inputs(H, W, B, term, ts)
    return oracle.evolve(img, phi0, term=term, g=g, ts=ts, iterations=iters,
                         reinit_period=period, early_stop_frac=frac)


def run_strips(comm, case, rank, world, steps=1, part=None):
    H, W, B, term, ts, iters, period, frac = case
    img, phi0, g = case_inputs(H, W, B, term, ts)
    if part is None:
        part = strips.partition(H, W, ts, rank, world, steps=steps)
    sl = slice(part.s0, part.s1)
    comp = OracleCompute(part, img[:, sl] if term == "region" else None,
                         g[sl] if g is not None else None, term=term, ts=ts)
    v, st = strips.evolve(comm, comp, part, phi0[sl].copy(), term=term, bands=B,
                          iterations=iters, reinit_period=period, early_stop_frac=frac)
    a, b = part.own
    return part, v[a:b], st, comp.calls


def compare(case, part, v_own, st):
    """Differences from the whole-image oracle: (max |v - v_ref| over the
    owned rows, mask disagreements, the statistics that differ)."""
    v_ref, m_ref, s_ref = whole_image(case)
    ref = v_ref[part.y0:part.y1]
    err = float(np.max(np.abs(v_own - ref)))
    bad_mask = int(np.count_nonzero((v_own >= 0) != (m_ref[part.y0:part.y1] == 1)))
    diff = [k for k in ("iterations_run", "last_flips", "area_plus") if st[k] != s_ref[k]]
    if case[3] == "region":
        if not np.allclose(st["c_plus"], s_ref["c_plus"], rtol=1e-12, atol=1e-14):
            diff.append("c_plus")
        if not np.allclose(st["c_minus"], s_ref["c_minus"], rtol=1e-12, atol=1e-14):
            diff.append("c_minus")
    return err, bad_mask, diff, int(s_ref["iterations_run"])


# ---------------------------------------------------------------- partition
@pytest.mark.parametrize("H,world,ts,steps", [(37, 2, 9, 1), (37, 3, 9, 1), (100, 7, 15, 1),
                                               (10, 2, 3, 1), (37, 3, 9, 2), (100, 4, 7, 3)])
def test_partition_covers_rows_once(H, world, ts, steps):
    parts = [strips.partition(H, 17, ts, r, world, steps=steps) for r in range(world)]
    h = strips.halo_rows(ts, steps)
    assert parts[0].y0 == 0 and parts[-1].y1 == H
    for p, q in zip(parts, parts[1:]):
        assert p.y1 == q.y0
    sizes = [p.y1 - p.y0 for p in parts]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= h
    for r, p in enumerate(parts):
        assert p.halo == h == steps * ((ts - 1) // 2 + 1) and p.steps == steps
        assert p.s0 == max(0, p.y0 - h) and p.s1 == min(H, p.y1 + h)
        assert (p.y0, p.y1) == strips.owned_rows(H, r, world)
        a, b = p.own
        assert b - a == p.y1 - p.y0 and p.rows == p.s1 - p.s0


def test_partition_refuses_thin_strips():
    with pytest.raises(ValueError):
        strips.partition(9, 8, 9, 0, 2)            # 4 rows a rank, halo 5
    with pytest.raises(ValueError):
        strips.partition(20, 8, 9, 2, 2)
    with pytest.raises(ValueError):
        strips.partition(37, 8, 9, 0, 3, steps=3)  # 12 rows a rank, halo 15
    with pytest.raises(ValueError):
        strips.partition(37, 8, 9, 0, 2, steps=0)


def test_reinit_schedule():
    assert [strips.reinit_after(n, 1) for n in range(4)] == [True] * 4
    assert [strips.reinit_after(n, 0) for n in range(4)] == [False] * 4
    assert [strips.reinit_after(n, 3) for n in range(7)] == [False, False, True, False, False,
                                                              True, False]


# ---------------------------------------------------------------- one rank
@pytest.mark.parametrize("case", CASES)
def test_one_rank_is_the_whole_image(case):
    part, v, st, calls = run_strips(strips.LocalComm(), case, 0, 1)
    assert (part.s0, part.s1) == (0, case[0])
    err, bad, diff, n_ref = compare(case, part, v, st)
    assert diff == [] and bad == 0 and err < 1e-9, (err, bad, diff)
    # one step and one partials pass per iteration, one more partials pass
    # for phi0; the normaliser pass only for vector images
    assert calls["step"] == n_ref and calls["partials"] == n_ref + 1
    assert calls["dmax"] == (n_ref if case[2] > 1 else 0)
    if case[7] > 0:
        assert 1 < n_ref < case[5]                  # the early stop ends it midway


# ---------------------------------------------------------------- gloo ranks
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_1409_7474_gb300 import strips as S
    res = {}
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        comm = S.TorchComm()
        # the exchange itself: rank-coded rows arrive from the right side
        part = S.partition(40, 6, 5, rank, world)
        v = np.full((part.rows, 6), float(rank), dtype=np.float32)
        a, b = part.own
        v[a:b] += np.arange(b - a, dtype=np.float32)[:, None] * 0.001
        v = S.exchange_halo(comm, part, v, binary=False)
        res["halo_top"] = None if a == 0 else v[:a, 0].tolist()
        res["halo_bottom"] = None if b == part.rows else v[b:, 0].tolist()
        res["own"] = (part.y0, part.y1, a, b)
        for i, case in enumerate(CASES):
            from test_strips import compare, run_strips
            p, v_own, st, _ = run_strips(comm, case, rank, world)
            res[i] = compare(case, p, v_own, st)
            if i == 0:
                # rank 0 gathers the owned rows into the whole image
                strip = np.zeros((p.rows, p.W))
                a, b = p.own
                strip[a:b] = v_own
                full = S.gather_rows(comm, p, strip)
                if rank == 0:
                    from test_strips import whole_image
                    res["gathered_err"] = float(np.max(np.abs(full - whole_image(case)[0])))
                else:
                    res["gathered_none"] = full is None
        # halos k steps deep, exchanged after every k-th step: the owned rows
        # stay the whole image's (k = 2 for every case; k = 3 where each
        # rank owns 3 (r + 1) rows)
        # Each case runs in full and stopped after 3 iterations, before
        # re-initialisation can wash out an error next to a cut
        for i, case in enumerate(CASES):
            short = case[:5] + (min(case[5], 3),) + case[6:]
            for k in (2, 3):
                if case[0] // world >= k * ((case[4] - 1) // 2 + 1):
                    for tag, c in (("full", case), ("short", short)):
                        p, v_own, st, calls = run_strips(comm, c, rank, world, steps=k)
                        res[("steps", i, k, tag)] = compare(c, p, v_own, st)
        # the exchanges a k-step run makes: one after every k-th step
        sent = []
        real_exchange = comm.exchange
        comm.exchange = lambda *args: sent.append(1) or real_exchange(*args)
        try:
            for k in (1, 2, 3):
                sent.clear()
                run_strips(comm, CASES[3][:5] + (7, 1, 0.0), rank, world, steps=k)
                res[("exchanges", k)] = len(sent)
        finally:
            comm.exchange = real_exchange
        # k steps between exchanges over a halo one step deep: rows next to
        # a cut go wrong.  The case that re-initialises every third step,
        # stopped after 3 iterations: the stale rows' values, not only their
        # signs, reach the owned rows, and the later re-initialisations
        # would wash the error out again
        import dataclasses
        c = CASES[1][:5] + (3,) + CASES[1][6:]
        p1 = S.partition(c[0], c[1], c[4], rank, world)
        p, v_own, st, _ = run_strips(comm, c, rank, world, part=dataclasses.replace(p1, steps=2))
        res["shallow"] = compare(c, p, v_own, st)
        # a driver whose halo exchange does nothing
        real = S.exchange_halo
        S.exchange_halo = lambda comm, part, v, binary: v
        try:
            p, v_own, st, _ = run_strips(comm, CASES[0], rank, world)
            res["no_halo"] = compare(CASES[0], p, v_own, st)
        finally:
            S.exchange_halo = real
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which fails the test
        res["error"] = repr(e)
    out.put((rank, res))


def _run_world(world):
    import torch.multiprocessing as mp
    oracle.build()                       # one build before the ranks load it
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reproduce_the_whole_image(world):
    res = _run_world(world)
    for r in range(world):
        assert "error" not in res[r], res[r].get("error")
    # halo rows hold the neighbour's owned rows: its first rows below a cut,
    # its last rows above one
    for r in range(world):
        part = strips.partition(40, 6, 5, r, world)
        h = part.halo
        if r > 0:
            prev = strips.partition(40, 6, 5, r - 1, world)
            n_prev = prev.y1 - prev.y0
            want = [r - 1 + 0.001 * k for k in range(n_prev - h, n_prev)]
            np.testing.assert_allclose(res[r]["halo_top"], want, rtol=0, atol=1e-6)
        if r < world - 1:
            want = [r + 1 + 0.001 * k for k in range(h)]
            np.testing.assert_allclose(res[r]["halo_bottom"], want, rtol=0, atol=1e-6)
    for i, case in enumerate(CASES):
        for r in range(world):
            err, bad, diff, _ = res[r][i]
            assert diff == [] and bad == 0 and err < 1e-9, (case, r, err, bad, diff)
    assert res[0]["gathered_err"] < 1e-9
    assert all(res[r]["gathered_none"] for r in range(1, world))
    # k-step halos: every case at k = 2, the ones that fit at k = 3
    ks = sorted({key[2] for key in res[0] if isinstance(key, tuple) and key[0] == "steps"})
    assert ks == [2, 3]
    for r in range(world):
        assert [res[r][("exchanges", k)] for k in (1, 2, 3)] == [7, 3, 2]
    for key in res[0]:
        if isinstance(key, tuple) and key[0] == "steps":
            for r in range(world):
                err, bad, diff, _ = res[r][key]
                assert diff == [] and bad == 0 and err < 1e-9, (key, r, err, bad, diff)
    assert any(res[r]["shallow"][0] > 1e-3 or res[r]["shallow"][1] > 0 for r in range(world))
    # without the exchange the rows next to a cut go wrong
    assert any(res[r]["no_halo"][0] > 1e-3 or res[r]["no_halo"][1] > 0 for r in range(world))
