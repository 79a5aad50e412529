"""Host logic of the continuous-batching server (serve.Server) on the CPU: the batch calls of the C ABI,
the contexts and the CUDA stream/event are replaced by fakes that keep a step clock per batch and check,
at every call, what the device would rely on.  The server must admit in arrival order within the HBM
budget and the slot cap, step a batch only while a member still has steps left, remove a member only
after its own last step, retire requests that fail (or can never fit) without stalling the stream, and
free every context."""
import numpy as np
import pytest

from paper_2504_09118_gb300 import binding as B
from paper_2504_09118_gb300 import serve


class FakeBatch:
    def __init__(self, storage):
        self.storage, self.clock, self.members, self.chunks, self.retunes = storage, 0, {}, 0, 0


class FakeLib:
    """The batch calls the server makes, with the library's contract asserted."""
    FDTD_F32, FDTD_F16, FDTD_BF16 = B.FDTD_F32, B.FDTD_F16, B.FDTD_BF16
    FdtdError = B.FdtdError

    def __init__(self, budget, max_slots):
        self.budget, self.max_slots = budget, max_slots
        self.bytes = {}          # handle -> estimated bytes of a member
        self.peak_bytes = self.peak_members = 0
        self.removed = []

    def _members(self):
        return sum(len(b.members) for b in self.batches)

    def fdtd_batch_create(self, storage, stream):
        b = FakeBatch(storage)
        self.batches = getattr(self, "batches", []) + [b]
        return b

    def fdtd_batch_set_tuning(self, b, **kw):
        b.tuning = kw

    def fdtd_batch_add(self, b, h):
        assert h.storage == b.storage and h not in b.members
        b.members[h] = [b.clock, None]
        self.bytes[h] = h.est
        self.peak_bytes = max(self.peak_bytes, sum(self.bytes.values()))
        self.peak_members = max(self.peak_members, self._members())

    def fdtd_batch_set_steps(self, b, h, n):
        assert b.members[h][1] is None and n >= 1
        b.members[h][1] = n

    def fdtd_batch_steps_done(self, b):
        return b.clock

    def fdtd_batch_step(self, b, K):
        # only while some member still has steps left
        assert any(b.clock - j < n for j, n in b.members.values())
        b.clock += K
        b.chunks += 1

    def fdtd_batch_remove(self, b, h):
        joined, n = b.members.pop(h)
        assert b.clock - joined >= n, "member removed before its last step"
        self.bytes.pop(h)
        self.removed.append((h.rid, b.clock - joined, n))

    def fdtd_batch_retune(self, b, trial):
        b.retunes += 1
        return {"kernel": 3, "tile_y": 16, "stages": 4}, 1.0, False

    def fdtd_batch_sync(self, b):
        pass

    def fdtd_batch_destroy(self, b):
        assert not b.members


class FakeCavity:
    live = 0
    fail_create = set()     # (nx, ny, nz) whose creation fails as if out of memory
    fail_load = set()       # ... whose set_fields fails

    def __init__(self, nx, ny, nz, dt, dx, ce, ch, storage, stream, order=2):
        if (nx, ny, nz) in FakeCavity.fail_create:
            raise B.FdtdError(B.FDTD_ERR_OOM, "out of device memory")
        self.handle = self
        self.storage, self.dims = storage, (nx, ny, nz)
        self.est = serve.device_bytes_estimate(nx, ny, nz, storage, ce is not None)
        self.rid = None
        FakeCavity.live += 1

    def set_fields(self, f, on_device=False):
        if self.dims in FakeCavity.fail_load:
            raise B.FdtdError(B.FDTD_ERR_ARG, "bad fields")

    def energy(self):
        return float(np.prod(self.dims))

    def get_fields(self):
        return []

    def close(self):
        FakeCavity.live -= 1


class FakeEvent:
    def record(self, stream=None):
        pass

    def synchronize(self):
        pass


class VirtualClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4
        return self.t

    def sleep(self, s):
        self.t += max(s, 1e-4)


@pytest.fixture
def fake_server(monkeypatch):
    import torch

    def make(budget, max_slots, **kw):
        lib = FakeLib(budget, max_slots)
        monkeypatch.setattr(serve, "B", lib)
        monkeypatch.setattr(serve, "Cavity", FakeCavity)
        monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: object())
        monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
        clock = VirtualClock()
        monkeypatch.setattr(serve.time, "sleep", clock.sleep)
        FakeCavity.live = 0
        FakeCavity.fail_create, FakeCavity.fail_load = set(), set()
        srv = serve.Server(0.1, hbm_budget_bytes=budget, max_slots=max_slots, K=16, **kw)
        return srv, lib, clock
    return make


def _requests(seed, n):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(0.002, n))
    return [serve.Request(i, float(t[i]), int(rng.integers(8, 41)), int(rng.integers(8, 41)),
                          int(rng.integers(8, 41)), int(rng.integers(5, 201)), bool(rng.integers(0, 2)),
                          fields=[np.zeros(1)]) for i in range(n)]


@pytest.mark.timeout(120)
def test_admission_budget_slots_and_exact_steps(fake_server, monkeypatch):
    reqs = _requests(7, 80)
    big = serve.device_bytes_estimate(40, 40, 40, B.FDTD_F32)
    budget, slots = 3 * big, 5
    srv, lib, clock = fake_server(budget, slots)
    # failure injection: one creation and one load fail; one request can never fit the budget
    reqs[10].nx, reqs[10].ny, reqs[10].nz = 13, 17, 19
    FakeCavity.fail_create.add((13, 17, 19))
    reqs[20].nx, reqs[20].ny, reqs[20].nz = 11, 23, 29
    FakeCavity.fail_load.add((11, 23, 29))
    reqs[30].nx, reqs[30].ny, reqs[30].nz = 400, 400, 400
    orig_init = FakeCavity.__init__

    def tagged_init(self, nx, ny, nz, *a, **kw):   # the request a context belongs to: the first unadmitted
        orig_init(self, nx, ny, nz, *a, **kw)       # one of its size (admission is in arrival order)
        self.rid = next(r.id for r in reqs if (r.nx, r.ny, r.nz) == (nx, ny, nz) and np.isnan(r.t_admit))
    monkeypatch.setattr(FakeCavity, "__init__", tagged_init)
    stats = srv.run(reqs, clock=clock)
    failed = sorted(r.id for r in reqs if r.error)
    assert failed == [10, 20, 30]
    assert stats.failed == 3 and stats.n == len(reqs) - 3
    # every other request ran exactly its own steps (removal asserts none left early) and has a result
    done = {rid: (taken, n) for rid, taken, n in lib.removed}
    assert sorted(done) == sorted(r.id for r in reqs if not r.error)
    for r in reqs:
        if not r.error:
            assert done[r.id][1] == r.steps and done[r.id][0] < r.steps + 2 * srv.K
            assert r.result == float(r.nx * r.ny * r.nz)
    # budget and slot cap held at every admission; admission in arrival order, never before arrival
    assert lib.peak_bytes <= budget and lib.peak_members <= slots and stats.max_active <= slots
    order = sorted(reqs, key=lambda r: r.arrival_s)
    adm = [r.t_admit for r in order]
    assert all(a <= b for a, b in zip(adm, adm[1:]))
    assert all(r.t_admit >= r.arrival_s for r in reqs)
    assert all(r.t_done >= r.t_admit for r in reqs)
    # nothing left behind
    assert srv.used == 0 and not srv.active and FakeCavity.live == 0
    srv.close()


@pytest.mark.timeout(60)
def test_request_over_the_whole_budget_does_not_stall(fake_server):
    srv, lib, clock = fake_server(10 << 20, 4)
    reqs = [serve.Request(0, 0.0, 300, 300, 300, 50, fields=[np.zeros(1)])]
    stats = srv.run(reqs, clock=clock)
    assert stats.n == 0 and stats.failed == 1 and "budget" in reqs[0].error
    srv.close()


@pytest.mark.timeout(60)
def test_retune_only_after_membership_changes(fake_server):
    srv, lib, clock = fake_server(1 << 34, 8, retune=True)
    reqs = [serve.Request(0, 0.0, 16, 16, 16, 100, fields=[np.zeros(1)])]
    srv.run(reqs, clock=clock)
    f32 = lib.batches[0]
    assert f32.chunks == 7            # ceil(100 / 16) chunks, then the member is removed
    assert f32.retunes == 1 and srv.retunes["model"] == 1
    srv.close()


def test_bad_configuration_is_rejected(fake_server):
    for kw in (dict(budget=0, max_slots=4), dict(budget=1 << 30, max_slots=0)):
        with pytest.raises(ValueError):
            fake_server(kw["budget"], kw["max_slots"])
