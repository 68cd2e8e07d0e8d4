"""Row strips on the GPU through lse_strip_partials / _dmax / _step.

The strip driver runs with the library's compute; its ranks are host
threads of one process, each with its own context, meeting at host-side
barriers for the all-reduce and the halo exchange (no kernel of one rank
waits on another's).  Checks:

* the partial sums of any rows are the exact fixed-point sums (each band
  value rounded once to a multiple of 2^-k) and the counts of the plain
  definitions;
* one strip step with given totals is the oracle's step with the same
  statistics;
* the evolution split over 2 or 3 ranks gives the bits of the unsplit
  (one-rank) run -- the integer totals do not depend on the split -- and
  agrees with lse_evolve on the whole image and with the oracle within the
  parity tolerances.
"""
import threading

import numpy as np
import pytest

import oracle
from _parity import assert_mask_parity
from paper_1409_7474_gb300 import scenes, strips

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def lse():
    import paper_1409_7474_gb300.lse as m
    return m


def torch_max(a, b):
    import torch
    return torch.maximum(a, b)


class ThreadComm:
    """Ranks as threads of one process: all-reduce and neighbour exchange
    through shared slots and a barrier (timed, so a failing rank fails the
    test instead of stalling it)."""

    class World:
        def __init__(self, n):
            self.n = n
            self.barrier = threading.Barrier(n, timeout=120)
            self.slots = {}

    def __init__(self, world, rank):
        self.w = world
        self.rank = rank
        self.world = world.n

    def all_reduce(self, values, op):
        self.w.slots[("r", self.rank)] = np.array(values, copy=True)
        self.w.barrier.wait()
        vals = [self.w.slots[("r", r)] for r in range(self.world)]
        self.w.barrier.wait()
        out = vals[0].copy()
        for v in vals[1:]:
            out = out + v if op == "sum" else np.maximum(out, v)
        return out

    def all_reduce_tensor(self, t, op):
        self.w.slots[("t", self.rank)] = t.clone()
        self.w.barrier.wait()
        vals = [self.w.slots[("t", r)] for r in range(self.world)]
        self.w.barrier.wait()
        acc = vals[0].clone()
        for v in vals[1:]:
            acc = acc + v if op == "sum" else torch_max(acc, v)
        t.copy_(acc)
        return t

    def exchange(self, to_prev, to_next, like_prev, like_next):
        if to_prev is not None:
            self.w.slots[("x", self.rank, self.rank - 1)] = to_prev.clone()
        if to_next is not None:
            self.w.slots[("x", self.rank, self.rank + 1)] = to_next.clone()
        self.w.barrier.wait()
        got_prev = self.w.slots.get(("x", self.rank - 1, self.rank)) if to_prev is not None \
            else None
        got_next = self.w.slots.get(("x", self.rank + 1, self.rank)) if to_next is not None \
            else None
        self.w.barrier.wait()
        return got_prev, got_next


def run_split(torch, lse, world, img, phi0, g, term, ts, iterations, period, frac,
              device_sums=None, steps=1):
    """The strip driver over `world` thread ranks, halos `steps` steps deep;
    returns the whole v (owned rows stacked) and rank 0's statistics."""
    B = img.shape[0] if img is not None else 1
    H, W = phi0.shape
    w = ThreadComm.World(world)
    out, errors = {}, []
    parts = [strips.partition(H, W, ts, r, world, steps=steps) for r in range(world)]
    ctxs = [lse.Context(0, max_pixels=parts[r].rows * W, max_bands=max(B, 1))
            for r in range(world)]

    def rank_main(r):
        try:
            part = parts[r]
            sl = slice(part.s0, part.s1)
            dimg = torch.from_numpy(np.ascontiguousarray(img[:, sl])).cuda() \
                if term == "region" else None
            dg = torch.from_numpy(np.ascontiguousarray(g[sl])).cuda() if g is not None else None
            comp = strips.LibraryCompute(ctxs[r], part, dimg, dg, term=term, ts=ts,
                                         device_sums=device_sums)
            p0 = torch.from_numpy(np.ascontiguousarray(phi0[sl])).cuda()
            v, st = strips.evolve(ThreadComm(w, r), comp, part, p0, term=term, bands=B,
                                  iterations=iterations, reinit_period=period,
                                  early_stop_frac=frac)
            torch.cuda.synchronize()
            a, b = part.own
            out[r] = (v[a:b].cpu().numpy(), st)
        except Exception as e:  # reported below
            errors.append(repr(e))
            w.barrier.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    for c in ctxs:
        c.destroy()
    assert not errors, errors
    v = np.concatenate([out[r][0] for r in range(world)])
    return v, out[0][1], [out[r][1] for r in range(world)]


CASES = [
    # (H, W, B, term, ts, iterations, reinit_period, early_stop_frac)
    (300, 260, 1, "region", 9, 40, 1, 0.0),
    (257, 200, 3, "region", 9, 30, 1, 0.0),
    (270, 190, 1, "edge", 9, 40, 1, 0.0),
    (301, 244, 1, "region", 7, 30, 3, 0.0),
    (280, 256, 1, "region", 9, 200, 1, 4e-3),
]


def case_inputs(H, W, B, term):
    img, _, _ = scenes.rect_scene(H, W, W // 2, H // 3, noise=0.06, seed_pos=H, seed_noise=W)
    img = np.concatenate([img * (1.0 - 0.2 * b) + 0.1 * b for b in range(B)]).astype(np.float32)
    if term == "edge":
        phi0 = scenes.box_phi(H, W, [(4, 4, H - 4, W - 4)])
    else:
        phi0 = scenes.circle_phi(H, W, cy=H * 0.45, cx=W * 0.55, radius=min(H, W) / 3.5)
    return img, phi0.astype(np.float32)


@pytest.mark.parametrize("case", CASES)
def test_split_runs_agree(torch, lse, case):
    H, W, B, term, ts, iters, period, frac = case
    img, phi0 = case_inputs(H, W, B, term)
    g = None
    if term == "edge":
        with lse.Context(0, max_pixels=H * W, max_bands=B) as c:
            g = c.precompute_edge(torch.from_numpy(img).cuda(), 1.0, 9, 255.0).cpu().numpy()
    runs = {n: run_split(torch, lse, n, img, phi0, g, term, ts, iters, period, frac)
            for n in (1, 2, 3)}
    v1, st1, _ = runs[1]
    # the statistics kept on the host (one round trip per iteration) give
    # the same bits as the device-resident record
    runs["host"] = run_split(torch, lse, 2, img, phi0, g, term, ts, iters, period, frac,
                             device_sums=False)
    assert np.array_equal(runs["host"][0].view(np.uint32), v1.view(np.uint32))
    # halos two and three steps deep, exchanged after every second / third step
    for n, k in ((2, 2), (3, 3)):
        runs[(n, k)] = run_split(torch, lse, n, img, phi0, g, term, ts, iters, period, frac,
                                 steps=k)
    for n in (2, 3, (2, 2), (3, 3)):
        vn, stn, all_st = runs[n]
        # the bits of the unsplit run, and the same statistics on every rank
        assert np.array_equal(vn.view(np.uint32), v1.view(np.uint32)), n
        for s in all_st:
            for k in ("iterations_run", "last_flips", "area_plus"):
                assert s[k] == st1[k], (n, k)
    # the whole image through lse_evolve (its statistics are summed per tile
    # in another grouping: agreement within the parity tolerances)
    with lse.Context(0, max_pixels=H * W, max_bands=B) as c:
        x = torch.from_numpy(img).cuda()
        dg = torch.from_numpy(g).cuda() if g is not None else None
        ve, me, se = c.evolve(x if term == "region" else None, torch.from_numpy(phi0).cuda(),
                              term, g=dg, ts=ts, iterations=iters, reinit_period=period)
    assert_mask_parity(v1 >= 0, me.cpu().numpy())
    # the FP64 oracle on the whole image
    g64 = g.astype(np.float64) if g is not None else None
    v_ref, m_ref, s_ref = oracle.evolve(img.astype(np.float64), phi0.astype(np.float64),
                                        term=term, g=g64, ts=ts, iterations=iters,
                                        reinit_period=period)
    assert_mask_parity(v1 >= 0, m_ref)
    assert st1["iterations_run"] == s_ref["iterations_run"]


@pytest.mark.parametrize("W,B", [(61, 3), (64, 3), (64, 1), (68, 5)])
def test_partials_are_exact_fixed_point_sums(torch, lse, W, B):
    # W a multiple of 4: the pass reads four columns a thread (16-byte loads)
    H = 97
    rng = np.random.default_rng(5)
    img = rng.uniform(-2.0, 3.0, (B, H, W)).astype(np.float32)
    phi = rng.normal(size=(H, W)).astype(np.float32)
    prev = rng.normal(size=(H, W)).astype(np.float32)
    k = lse.strip_scale(float(np.abs(img).max()), H * W)
    with lse.Context(0, max_pixels=H * W, max_bands=B) as c:
        for rows in [(0, H), (10, 11), (13, 80), (96, 97), (40, 40)]:
            for place in ("device", "host"):
                args = [img, phi, prev]
                if place == "device":
                    args = [torch.from_numpy(a).cuda() for a in args]
                s = c.strip_partials(args[0], args[1], rows[0], rows[1], k, args[2])
                y0, y1 = rows
                I = img[:, y0:y1].astype(np.float64)
                q = np.sign(I) * np.floor(np.abs(I) * 2.0 ** k + 0.5)   # nearest, ties away
                plus = phi[y0:y1] >= 0
                w = np.where(plus, 1, -1)
                assert s.npix == (y1 - y0) * W
                assert s.n_plus == int(plus.sum())
                assert s.flips == int(np.count_nonzero(plus != (prev[y0:y1] >= 0)))
                for b in range(B):
                    qi = q[b].astype(np.int64)
                    assert s.sum_a[b] == int(qi.sum())
                    assert s.sum_w[b] == int((w * qi).sum())
                if y1 > y0:
                    assert s.imin == float(img[0, y0:y1].min())
                    assert s.imax == float(img[0, y0:y1].max())
                    assert s.amax == float(np.abs(img[:, y0:y1]).max())
        # phi NULL: only the range
        s = c.strip_partials(torch.from_numpy(img).cuda(), None, 0, H)
        assert s.n_plus == 0 and s.sum_a[0] == 0 and s.imax == float(img[0].max())
        # a NaN in the owned rows is reported
        bad = img.copy()
        bad[B - 1, 50, 7] = np.nan
        with pytest.raises(lse.LseError) as e:
            c.strip_partials(torch.from_numpy(bad).cuda(), torch.from_numpy(phi).cuda(), 40, 60,
                             k)
        assert e.value.status == lse.LSE_ERR_NONFINITE


@pytest.mark.parametrize("B,term", [(1, "region"), (3, "region"), (1, "edge")])
def test_one_strip_step_is_the_oracle_step_with_the_same_statistics(torch, lse, B, term):
    H, W, ts = 150, 133, 9
    img, phi = case_inputs(H, W, B, "region")
    rng = np.random.default_rng(9)
    phi = (phi + 0.3 * rng.normal(size=phi.shape)).astype(np.float32)
    part = strips.partition(H, W, ts, 1, 3)         # a middle strip
    sl = slice(part.s0, part.s1)
    a, b = part.own
    with lse.Context(0, max_pixels=H * W, max_bands=B) as c:
        x = torch.from_numpy(img).cuda()
        g = c.precompute_edge(x, 1.0, 9, 255.0) if term == "edge" else None
        # the whole image's totals, from the partials of all its rows
        k = lse.strip_scale(float(np.abs(img).max()), H * W)
        tot = c.strip_partials(x, torch.from_numpy(phi).cuda(), 0, H, k)
        tot.npix = H * W
        xs = torch.from_numpy(np.ascontiguousarray(img[:, sl])).cuda()
        ps = torch.from_numpy(np.ascontiguousarray(phi[sl])).cuda()
        norm = 0.0
        if term == "region" and B > 1:
            norm = max(c.strip_dmax(xs, a, b, tot), 0.0)
            # the maximum over all rows bounds the strip's
            assert c.strip_dmax(x, 0, H, tot) >= norm
            norm = c.strip_dmax(x, 0, H, tot)
        v = c.strip_step(xs if term == "region" else None, ps, tot if term == "region" else None,
                         norm, term, g=g[sl].contiguous() if g is not None else None, ts=ts)
        v = v.cpu().numpy()
    T = strips.Totals(npix=H * W, n_plus=tot.n_plus, sum_w=np.array(tot.sum_w[:B]),
                      sum_a=np.array(tot.sum_a[:B]), imin=tot.imin, imax=tot.imax,
                      fix_k=tot.fix_k, bands=B)
    cp, cm = strips.means(T)
    img64 = img.astype(np.float64)
    if term == "edge":
        v_ref = oracle.step_given(img64[:, sl], phi[sl].astype(np.float64), [0.0], [0.0], 0.0,
                                  term="edge", g=g[sl].cpu().numpy().astype(np.float64), ts=ts)
    else:
        if B == 1:
            d = cp[0] - cm[0]
            M = max(abs(d * (2.0 * tot.imax - cp[0] - cm[0])),
                    abs(d * (2.0 * tot.imin - cp[0] - cm[0])))
        else:
            D = sum((cp[j] - cm[j]) * (2.0 * img64[j] - cp[j] - cm[j]) for j in range(B))
            M = float(np.abs(D).max())
            assert abs(M - norm) <= 1e-5 * M          # FP32 D on the GPU
        v_ref = oracle.step_given(img64[:, sl], phi[sl].astype(np.float64), cp, cm, M,
                                  ts=ts)
    err = np.abs(v[a:b] - v_ref[a:b])
    assert err.max() <= 2e-5 * (1.0 + np.abs(v_ref[a:b]).max()), err.max()


def test_strip_step_rejects_bad_arguments(torch, lse):
    with lse.Context(0, max_pixels=64 * 64, max_bands=1) as c:
        x = torch.rand(1, 32, 32, device="cuda")
        p = torch.rand(32, 32, device="cuda") - 0.5
        tot = c.strip_partials(x, p, 0, 32, 40)
        with pytest.raises(lse.LseError):           # the region term needs totals
            c.strip_step(x, p, None, 0.0, "region")
        with pytest.raises(lse.LseError):           # rows outside the strip
            c.strip_partials(x, p, 5, 40, 40)
        bad = lse.StripSums.from_buffer_copy(tot)
        bad.n_plus = bad.npix + 1
        with pytest.raises(lse.LseError):
            c.strip_step(x, p, bad, 0.0, "region")
        with pytest.raises(lse.LseError):           # dt must be positive
            c.strip_dmax(x, 0, 32, tot, dt=-1.0)


def test_device_records_defer_their_conditions_to_strip_status(torch, lse):
    # partial sums written into device memory return at once; a NaN they met
    # is reported by lse_strip_status (once), as is nothing for clean data
    H, W = 64, 64
    rng = np.random.default_rng(3)
    img = rng.uniform(0.0, 1.0, (1, H, W)).astype(np.float32)
    phi = rng.normal(size=(H, W)).astype(np.float32)
    with lse.Context(0, max_pixels=H * W, max_bands=1) as c:
        rec = torch.empty(lse.STRIP_SUMS_WORDS, dtype=torch.int64, device="cuda")
        x = torch.from_numpy(img).cuda()
        p = torch.from_numpy(phi).cuda()
        c.strip_partials(x, p, 0, H, 40, out=rec)
        c.strip_status()
        host = c.strip_partials(x, p, 0, H, 40)
        words = rec.cpu().numpy()
        assert words[0] == H * W and words[1] == host.n_plus and words[3] == host.sum_w[0]
        bad = img.copy()
        bad[0, 10, 10] = np.inf
        c.strip_partials(torch.from_numpy(bad).cuda(), p, 0, H, 40, out=rec)
        with pytest.raises(lse.LseError) as e:
            c.strip_status()
        assert e.value.status == lse.LSE_ERR_NONFINITE
        c.strip_status()                   # reported once
