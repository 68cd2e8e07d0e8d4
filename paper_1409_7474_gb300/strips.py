"""Row-strip decomposition of one evolution over several processes.

One image, one evolution, one process per GPU: rank ``i`` of ``world`` owns a
band of consecutive rows and holds them together with ``h = r + 1`` halo
rows on each cut side (``r = (ts - 1) // 2``).  Eq. 18's central differences
reach one row and Step 4's smoothing ``r`` rows, so a step on the strip gives
the owned rows of the whole image's step exactly, provided every rank uses
the whole image's statistics: the means of Eq. 15 and, for vector images,
the normaliser of Eq. 17 are global.  Per iteration the driver therefore

* adds the ranks' partial statistics of the current LSF -- ``|P|``, the sign
  changes of the last step and ``sum_P I_b`` per band: ``B + 2`` numbers, one
  all-reduce (the edge term needs the two counts only);
* for vector images takes the maximum of the ranks' ``max |D|`` (a second,
  one-number all-reduce);
* steps every strip with the totals, and
* copies each strip's first and last ``h`` owned rows into its neighbours'
  halo rows (only the sign when the next step re-initialises: one byte a
  pixel).

With an exchange period of ``k`` steps (``partition(..., steps=k)``) the
halo is ``h = k (r + 1)`` rows deep and the copy runs after every ``k``-th
step only.  Each step spoils the ``r + 1`` rows next to a cut it cannot see
past, so ``k`` steps leave the owned rows exact (temporal blocking of the
halo).  Each exchange then carries ``k`` times the rows, but there are
``1 / k`` as many; the ranks compute ``2 (k - 1) (r + 1)`` more rows a step.
The statistics stay per iteration: they come from the owned rows.

Once per evolution it also reduces the image's range (the one-band
normaliser's closed form and the fixed-point scale) and ``sum I_b``.

The driver does no arithmetic of the method.  A *compute* object does it for
one strip: :class:`LibraryCompute` calls the CUDA library's ``lse_strip_*``
entries; any object with the same methods (``range``, ``scale``,
``partials``, ``dmax``, ``step``) can stand in for it.  The communicator
wraps ``torch.distributed`` (NCCL for CUDA buffers, gloo on CPU); halos go
by point-to-point send and receive into each GPU's own memory.

With one band or the edge term, ``LibraryCompute`` keeps the statistics in
device memory (``device_sums``): the partial sums are written into a device
record, the ranks add its integer words on the device, and the next step
reads it in stream order, so an iteration enqueues its work without waiting
on the host (the early stop, when on, reads the sign-change count each
iteration).  Vector images take the host path: each step's max |D| is a
second reduction over the ranks.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

try:
    import torch
except ImportError:  # the driver itself only needs numpy
    torch = None


# ---------------------------------------------------------------- partition
@dataclass(frozen=True)
class Partition:
    """Rows of rank ``rank``: it owns image rows [y0, y1) and holds the strip
    [s0, s1) (owned rows plus ``halo`` rows on each side, clipped to the
    image).  ``steps``: steps between halo exchanges (the halo is that many
    steps deep)."""
    H: int
    W: int
    rank: int
    world: int
    halo: int
    y0: int
    y1: int
    s0: int
    s1: int
    steps: int = 1

    @property
    def rows(self) -> int:
        """Rows of the strip."""
        return self.s1 - self.s0

    @property
    def own(self) -> tuple[int, int]:
        """The owned rows as strip rows [a, b)."""
        return self.y0 - self.s0, self.y1 - self.s0


def halo_rows(ts: int, steps: int = 1) -> int:
    """Halo rows a strip needs for template size ts to take ``steps`` steps
    between exchanges: steps (r + 1)."""
    return int(steps) * ((int(ts) - 1) // 2 + 1)


def owned_rows(H: int, rank: int, world: int) -> tuple[int, int]:
    """The image rows [y0, y1) rank ``rank`` owns: ``world`` runs of
    H // world or H // world + 1 rows, the longer ones first."""
    base, extra = divmod(int(H), int(world))
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def partition(H: int, W: int, ts: int, rank: int, world: int, steps: int = 1) -> Partition:
    """Splits H rows over ``world`` ranks (``owned_rows``) with halos deep
    enough for ``steps`` steps between exchanges.  Every rank must own at
    least the halo's rows, so that a halo comes from one neighbour."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if int(steps) < 1:
        raise ValueError(f"steps between exchanges must be at least 1, not {steps}")
    h = halo_rows(ts, steps)
    if int(H) // int(world) < h:
        raise ValueError(f"{H} rows over {world} ranks leave fewer than the {h} halo rows "
                         f"a rank must own (ts = {ts}, {steps} steps between exchanges)")
    y0, y1 = owned_rows(H, rank, world)
    return Partition(int(H), int(W), rank, world, h, y0, y1, max(0, y0 - h), min(H, y1 + h),
                     int(steps))


# ---------------------------------------------------------------- communicators
class LocalComm:
    """One rank: reductions and exchanges are identities."""
    rank = 0
    world = 1

    def all_reduce(self, values: np.ndarray, op: str) -> np.ndarray:
        return np.array(values, copy=True)

    def all_reduce_tensor(self, t, op: str):
        return t

    def exchange(self, to_prev, to_next, like_prev, like_next):
        return None, None


class TorchComm:
    """Collectives of ``torch.distributed``: the default process group, or
    ``group``.  With NCCL the reductions go through a small CUDA tensor on
    ``device``; halos stay on the device of the rows sent."""

    def __init__(self, group=None, device=None):
        import torch.distributed as dist
        self._dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self._nccl = dist.get_backend(group) == "nccl"
        self.device = device

    def _peer(self, r: int) -> int:
        if self.group is None:
            return r
        return self._dist.get_global_rank(self.group, r)

    def all_reduce(self, values: np.ndarray, op: str) -> np.ndarray:
        t = torch.from_numpy(np.ascontiguousarray(values))
        if self._nccl:
            t = t.to(self.device or torch.device("cuda", torch.cuda.current_device()))
        rop = {"sum": self._dist.ReduceOp.SUM, "max": self._dist.ReduceOp.MAX}[op]
        self._dist.all_reduce(t, op=rop, group=self.group)
        return t.cpu().numpy()

    def all_reduce_tensor(self, t, op: str):
        """In place on a tensor: on its device with NCCL, through the host
        otherwise."""
        rop = {"sum": self._dist.ReduceOp.SUM, "max": self._dist.ReduceOp.MAX}[op]
        if self._nccl or t.device.type == "cpu":
            self._dist.all_reduce(t, op=rop, group=self.group)
        else:
            h = t.cpu()
            self._dist.all_reduce(h, op=rop, group=self.group)
            t.copy_(h)
        return t

    def send(self, t, dst: int):
        """Blocking point-to-point send of tensor ``t`` to rank ``dst``."""
        self._dist.send(t, dst=self._peer(dst), group=self.group)

    def recv(self, t, src: int):
        """Blocking receive into tensor ``t`` from rank ``src``."""
        self._dist.recv(t, src=self._peer(src), group=self.group)

    def exchange(self, to_prev, to_next, like_prev, like_next):
        """Sends ``to_prev`` to rank - 1 and ``to_next`` to rank + 1 (None
        where there is no neighbour) and receives buffers shaped like
        ``like_prev`` / ``like_next`` from them."""
        d = self._dist
        ops, got_prev, got_next = [], None, None
        if to_prev is not None:
            got_prev = torch.empty_like(like_prev)
            ops.append(d.P2POp(d.isend, to_prev.contiguous(), self._peer(self.rank - 1),
                               self.group))
            ops.append(d.P2POp(d.irecv, got_prev, self._peer(self.rank - 1), self.group))
        if to_next is not None:
            got_next = torch.empty_like(like_next)
            ops.append(d.P2POp(d.isend, to_next.contiguous(), self._peer(self.rank + 1),
                               self.group))
            ops.append(d.P2POp(d.irecv, got_next, self._peer(self.rank + 1), self.group))
        if ops:
            for req in d.batch_isend_irecv(ops):
                req.wait()
        return got_prev, got_next


# ---------------------------------------------------------------- statistics
@dataclass
class Totals:
    """Statistics of the current LSF, summed over the ranks (the fields of
    ``lse_strip_sums``): pixel count, |{phi >= 0}|, sign changes of the last
    step, sum of s(x) I_b(x) (s = +1 where phi >= 0, else -1) and sum of
    I_b(x) per band, band 0's range, max |I_b|, and the fixed-point scale
    of the sums (integer sums: values x 2^fix_k; floating sums: fix_k 0)."""
    npix: int
    n_plus: int = 0
    flips: int = 0
    sum_w: np.ndarray = field(default_factory=lambda: np.zeros(0))
    sum_a: np.ndarray = field(default_factory=lambda: np.zeros(0))
    imin: float = 0.0
    imax: float = 0.0
    amax: float = 0.0
    fix_k: int = 0
    bands: int = 1


@dataclass
class Partials:
    """One rank's share of Totals over its owned rows (returned by the
    compute's ``partials``)."""
    n_plus: int
    flips: int
    sum_w: np.ndarray
    sum_a: np.ndarray


def reinit_after(n: int, period: int) -> bool:
    """Whether iteration n (0-based) ends with the re-initialisation to the
    binary LSF (Step 3): every iteration for period 1, never for 0, after
    iterations k-1, 2k-1, ... for period k."""
    if period == 1:
        return True
    if period <= 0:
        return False
    return (n + 1) % period == 0


def _reduce_partials(comm, p: Partials, with_sum_a: bool, tot: Totals) -> Totals:
    """One all-reduce of (|P|, flips, sum_w per band[, sum_a per band])."""
    B = len(p.sum_w)
    sw = np.asarray(p.sum_w)
    dt = np.int64 if sw.dtype.kind in "iu" else np.float64
    vec = [np.array([p.n_plus, p.flips], dtype=dt), sw.astype(dt)]
    if with_sum_a:
        vec.append(np.asarray(p.sum_a).astype(dt))
    got = comm.all_reduce(np.concatenate(vec), "sum")
    out = Totals(npix=tot.npix, n_plus=int(got[0]), flips=int(got[1]), sum_w=got[2:2 + B],
                 sum_a=got[2 + B:2 + 2 * B] if with_sum_a else tot.sum_a, imin=tot.imin,
                 imax=tot.imax, amax=tot.amax, fix_k=tot.fix_k, bands=tot.bands)
    return out


# ---------------------------------------------------------------- halo exchange
def exchange_halo(comm, part: Partition, v, binary: bool):
    """Overwrites the halo rows of strip ``v`` (Hs x W, torch tensor or
    numpy array) with the neighbours' first / last ``halo`` owned rows.
    ``binary``: the next step reads only the sign, so one byte a pixel
    travels (+1 / -1)."""
    if comm.world == 1:
        return v
    a, b = part.own
    h = part.halo
    is_np = isinstance(v, np.ndarray)
    t = torch.from_numpy(v) if is_np else v

    def pack(rows):
        if binary:
            return torch.where(rows >= 0, 1, -1).to(torch.int8)
        return rows.contiguous()

    to_prev = pack(t[a:a + h]) if part.rank > 0 else None
    to_next = pack(t[b - h:b]) if part.rank < part.world - 1 else None
    like = pack(t[a:a + h])
    got_prev, got_next = comm.exchange(to_prev, to_next, like, like)
    if got_prev is not None:
        t[:a] = got_prev.to(t.dtype)
    if got_next is not None:
        t[b:] = got_next.to(t.dtype)
    return t.numpy() if is_np else t


# ---------------------------------------------------------------- driver
def evolve(comm, compute, part: Partition, phi0, *, term: str = "region", bands: int = 1,
           iterations: int = 200, reinit_period: int = 1, early_stop_frac: float = 0.0):
    """Runs the evolution of one image split into row strips; every rank calls
    it with its own strip.

    phi0      the strip's rows [s0, s1) of the initial LSF (Hs x W; a torch
              tensor or numpy array of the compute's choosing).
    compute   the strip's arithmetic (LibraryCompute, or an object with its
              methods).
    Returns (v, stats): ``v`` is the strip (Hs x W) after the last executed
    step -- its owned rows, ``v[a:b]`` with ``(a, b) = part.own``, are the
    whole image's rows [y0, y1) -- and ``stats`` the statistics lse_evolve
    reports (iterations run, sign changes of the last step, |{v >= 0}|, and
    for the region term c+/c- of the returned LSF and the last normaliser),
    equal on every rank."""
    region = term == "region"
    B = int(bands) if region else 1
    npix = part.H * part.W
    tot = Totals(npix=npix, bands=B)
    if region:
        # once: band 0's range, max |I_b| and the scale of the integer sums
        lo, hi, am = compute.range()
        got = comm.all_reduce(np.array([-lo, hi, am], dtype=np.float64), "max")
        tot.imin, tot.imax, tot.amax = -float(got[0]), float(got[1]), float(got[2])
        tot.fix_k = int(compute.scale(tot.amax, npix))
    if getattr(compute, "device_sums", False):
        return _evolve_device(comm, compute, part, phi0, tot, region, B, iterations,
                              reinit_period, early_stop_frac)
    phi = phi0
    tot = _reduce_partials(comm, compute.partials(phi, None, tot.fix_k), True, tot)
    first_n_plus = tot.n_plus
    binarise_in = False
    norm = 0.0
    v = phi
    n_run = 0
    for n in range(int(iterations)):
        norm = 0.0
        if region and B > 1:
            d = compute.dmax(tot)
            norm = float(comm.all_reduce(np.array([d], dtype=np.float64), "max")[0])
        v = compute.step(phi, binarise_in, tot, norm)
        reinit = reinit_after(n, reinit_period)
        if (n + 1) % part.steps == 0:
            v = exchange_halo(comm, part, v, binary=reinit)
        tot = _reduce_partials(comm, compute.partials(v, phi, tot.fix_k), False, tot)
        n_run = n + 1
        phi = v
        binarise_in = reinit
        if early_stop_frac > 0.0 and tot.flips < early_stop_frac * npix:
            break
    stats = {"iterations_run": n_run, "last_flips": tot.flips, "area_plus": tot.n_plus,
             "initial_area_plus": first_n_plus, "totals": tot}
    if region:
        cp, cm = means(tot)
        stats.update(c_plus=list(cp), c_minus=list(cm), norm=norm)
    return v, stats


# words of a device lse_strip_sums record: npix, n_plus, flips, sum_w[8],
# sum_a[8] (integers the ranks add), then imin, imax, amax and fix_k | bands
_INT_WORDS = 19
_W_NPLUS, _W_FLIPS, _W_SW, _W_SA = 1, 2, 3, 11


def _evolve_device(comm, compute, part, phi0, tot, region, B, iterations, reinit_period,
                   early_stop_frac):
    """``evolve`` with the statistics kept in device memory: each iteration's
    partial sums go into a device record, the ranks add its integer words
    on the device (one all-reduce), the whole image's constants are written
    over the rest, and the next step reads the record in stream order -- no
    host round trip per iteration (but one to read the sign changes when
    the early stop is on)."""
    npix = tot.npix
    const = compute.constants(tot)

    def reduce(rec):
        comm.all_reduce_tensor(rec[:_INT_WORDS], "sum")
        rec[_INT_WORDS:] = const
        return rec

    phi = phi0
    rec = reduce(compute.partials_device(phi, None, tot.fix_k))
    first = rec
    binarise_in = False
    v = phi
    n_run = 0
    for n in range(int(iterations)):
        v = compute.step(phi, binarise_in, rec, 0.0)
        reinit = reinit_after(n, reinit_period)
        if (n + 1) % part.steps == 0:
            v = exchange_halo(comm, part, v, binary=reinit)
        rec = reduce(compute.partials_device(v, phi, tot.fix_k))
        n_run = n + 1
        phi = v
        binarise_in = reinit
        if early_stop_frac > 0.0 and int(rec[_W_FLIPS].item()) < early_stop_frac * npix:
            break
    words = rec.cpu().numpy()
    n_plus0 = int(first[_W_NPLUS].item())
    compute.finish()
    fin = Totals(npix=npix, n_plus=int(words[_W_NPLUS]), flips=int(words[_W_FLIPS]),
                 sum_w=words[_W_SW:_W_SW + B].copy(), sum_a=words[_W_SA:_W_SA + B].copy(),
                 imin=tot.imin, imax=tot.imax, amax=tot.amax, fix_k=tot.fix_k, bands=B)
    stats = {"iterations_run": n_run, "last_flips": fin.flips, "area_plus": fin.n_plus,
             "initial_area_plus": n_plus0, "totals": fin}
    if region:
        cp, cm = means(fin)
        stats.update(c_plus=list(cp), c_minus=list(cm), norm=0.0)
    return v, stats


def means(tot: Totals):
    """c+ and c- of Eq. 15 per band from the totals (0 for an empty side)."""
    scale = 2.0 ** -(tot.fix_k + 1)
    sw = np.asarray(tot.sum_w, dtype=np.float64)
    sa = np.asarray(tot.sum_a, dtype=np.float64)
    if np.asarray(tot.sum_w).dtype.kind in "iu":
        sp = np.array([float(int(x) + int(y)) for x, y in zip(tot.sum_a, tot.sum_w)]) * scale
        sm = np.array([float(int(x) - int(y)) for x, y in zip(tot.sum_a, tot.sum_w)]) * scale
    else:
        sp, sm = (sa + sw) / 2.0, (sa - sw) / 2.0
    n_minus = tot.npix - tot.n_plus
    cp = sp / tot.n_plus if tot.n_plus > 0 else np.zeros_like(sp)
    cm = sm / n_minus if n_minus > 0 else np.zeros_like(sm)
    return cp, cm


def gather_rows(comm, part: Partition, v):
    """Rank 0 receives every rank's owned rows and returns the whole H x W
    image (numpy); the other ranks return None."""
    a, b = part.own
    own = v[a:b]
    own_t = torch.from_numpy(np.ascontiguousarray(own)) if isinstance(own, np.ndarray) \
        else own.contiguous()
    if comm.world == 1:
        return own_t.cpu().numpy()
    if part.rank == 0:
        rows = [own_t.cpu()]
        for r in range(1, part.world):
            y0, y1 = owned_rows(part.H, r, part.world)
            buf = torch.empty((y1 - y0, part.W), dtype=own_t.dtype, device=own_t.device)
            comm.recv(buf, r)
            rows.append(buf.cpu())
        return torch.cat(rows).numpy()
    comm.send(own_t, 0)
    return None


# ---------------------------------------------------------------- the library's compute
class LibraryCompute:
    """One strip's arithmetic on the GPU through ``lse_strip_*``.

    image     region term: B x Hs x W (the strip's rows of the image, halo
              rows included), a CUDA tensor; None for the edge term.
    g         edge term: Hs x W rows of the whole image's g (Eq. 14).
    The LSF strips are CUDA float32 tensors."""

    def __init__(self, ctx, part: Partition, image=None, g=None, *, term: str = "region",
                 dt: float = 15.0, sigma: float = 1.0, ts: int = 9, device_sums=None):
        from . import lse
        self._lse = lse
        self.ctx = ctx
        self.part = part
        self.image = image
        self.g = g
        self.term = term
        self.dt, self.sigma, self.ts = float(dt), float(sigma), int(ts)
        self.bands = 1 if image is None or image.dim() == 2 else int(image.shape[0])
        # statistics in device memory (one band or the edge term: vector
        # images need each step's max |D| on the host)
        if device_sums is None:
            device_sums = term == "edge" or self.bands == 1
        self.device_sums = bool(device_sums) and (term == "edge" or self.bands == 1)

    def _sums(self, tot: Totals):
        s = self._lse.StripSums()
        s.npix, s.n_plus, s.flips = tot.npix, tot.n_plus, tot.flips
        for b in range(len(tot.sum_w)):
            s.sum_w[b] = int(tot.sum_w[b])
            s.sum_a[b] = int(tot.sum_a[b])
        s.imin, s.imax, s.amax = tot.imin, tot.imax, tot.amax
        s.fix_k, s.bands = tot.fix_k, tot.bands
        return s

    def range(self):
        a, b = self.part.own
        s = self.ctx.strip_partials(self.image, None, a, b)
        return s.imin, s.imax, s.amax

    def scale(self, amax: float, npix: int) -> int:
        return self._lse.strip_scale(amax, npix)

    def partials(self, phi, phi_prev, fix_k: int) -> Partials:
        a, b = self.part.own
        s = self.ctx.strip_partials(self.image, phi, a, b, fix_k, phi_prev,
                                    bands=self.bands)
        B = self.bands if self.term == "region" else 1
        return Partials(s.n_plus, s.flips, np.array(s.sum_w[:B], dtype=np.int64),
                        np.array(s.sum_a[:B], dtype=np.int64))

    def constants(self, tot: Totals):
        """The record's last four words for the whole image (imin, imax,
        amax, fix_k | bands << 32), on the LSF's device."""
        words = np.concatenate([
            np.array([tot.imin, tot.imax, tot.amax], dtype=np.float64).view(np.int64),
            np.array([tot.fix_k, tot.bands], dtype=np.int32).view(np.int64)])
        dev = self.image.device if self.image is not None else self.g.device
        return torch.from_numpy(words).to(dev)

    def partials_device(self, phi, phi_prev, fix_k: int):
        a, b = self.part.own
        rec = torch.empty(self._lse.STRIP_SUMS_WORDS, dtype=torch.int64, device=phi.device)
        return self.ctx.strip_partials(self.image, phi, a, b, fix_k, phi_prev,
                                       bands=self.bands, out=rec)

    def finish(self):
        self.ctx.strip_status()

    def dmax(self, tot: Totals) -> float:
        a, b = self.part.own
        return self.ctx.strip_dmax(self.image, a, b, self._sums(tot), self.dt)

    def step(self, phi, binarise_in: bool, tot, norm: float):
        if self.term == "region":
            rec = tot if torch is not None and isinstance(tot, torch.Tensor) else self._sums(tot)
            return self.ctx.strip_step(self.image, phi, rec, norm, "region",
                                       binarise_in=binarise_in, dt=self.dt,
                                       sigma=self.sigma, ts=self.ts)
        return self.ctx.strip_step(None, phi, None, 0.0, "edge", g=self.g,
                                   binarise_in=binarise_in, dt=self.dt, sigma=self.sigma,
                                   ts=self.ts)
