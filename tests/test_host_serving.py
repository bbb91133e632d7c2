"""Host logic of the continuous-batching request loop (serving.py), on the
CPU against a fake engine with the batch API's contract: first-in first-out
admission under the slot and memory budgets, a few iterations per tick,
retirement and reuse of memory, every request delivered once, and the
budget check."""
import pytest

torch = pytest.importorskip("torch")

from paper_2008_01440_gb300 import serving  # noqa: E402


class FakeEngine:
    def __init__(self, max_slots, budget):
        self.max_slots, self.free = max_slots, budget
        self.slots, self.next_id, self.iters, self.events = {}, 0, 0, []

    def close(self):
        self.events.append(("close",))


@pytest.fixture
def fake(monkeypatch):
    state = {}

    def create(max_slots, budget, kmax, stream=None, f64_apply=False):
        state["eng"] = FakeEngine(max_slots, budget)
        return state["eng"]

    def add(eng, nx, ny, nz, c0, cx, cy, cz, lmin, lmax, k, s, b, stream=None):
        n = nx * ny * nz
        if len(eng.slots) >= eng.max_slots or n > eng.free:
            return None
        sid = eng.next_id
        eng.next_id += 1
        eng.free -= n
        need = 2 + (n % 5) + k // 8          # iterations this system needs
        eng.slots[sid] = {"n": n, "left": need, "iters": 0, "rid": int(b[0].item())}
        eng.events.append(("add", int(b[0].item())))
        return sid

    def run(eng, tol, maxit, iter_limit=0, stream=None):
        for sl in eng.slots.values():
            step = min(iter_limit, sl["left"]) if iter_limit > 0 else sl["left"]
            sl["left"] -= step
            sl["iters"] += step
            eng.iters += step
        return sum(1 for sl in eng.slots.values() if sl["left"] > 0)

    def status(eng, sid):
        sl = eng.slots[sid]
        return sl["left"] <= 0, {"iters": sl["iters"], "status": 0, "true_relres": 0.0}

    def collect(eng, sid, x, stream=None):
        x.fill_(eng.slots[sid]["rid"])

    def release(eng, sid, stream=None):
        eng.free += eng.slots.pop(sid)["n"]
        eng.events.append(("release", sid))

    def stats(eng):
        return eng.iters, 7 * eng.iters

    for name, fn in (("pcg_batch_create", create), ("pcg_batch_add", add), ("pcg_batch_run", run),
                     ("pcg_batch_status", status), ("pcg_batch_collect", collect),
                     ("pcg_batch_release", release), ("pcg_batch_stats", stats)):
        monkeypatch.setattr(serving.nc, name, fn)
    return state


def requests(sizes, arrival=0.0):
    out = []
    for i, side in enumerate(sizes):
        out.append(serving.Request(rid=i, arrival=arrival, nx=side, ny=side, nz=side, c=(6.0, 1.0, 1.0, 1.0),
                                   lmin=0.1, lmax=2.0, k=8, s=1.001,
                                   b=torch.full((side ** 3,), float(i), dtype=torch.float64)))
    return out


def test_fifo_admission_under_budget_and_reuse(fake):
    sizes = [10, 12, 9, 11, 8, 12, 10]                 # 1000 .. 1728 unknowns
    reqs = requests(sizes)
    budget = 12 ** 3 + 10 ** 3                         # room for about two at a time
    stats = {}
    serving.serve_continuous(reqs, budget, max_slots=3, kmax=8, iters_per_tick=1, stats=stats)
    eng = fake["eng"]
    adds = [e[1] for e in eng.events if e[0] == "add"]
    assert adds == list(range(len(sizes)))             # admitted in arrival order
    assert all(r.t_done >= r.t_admit >= r.arrival for r in reqs)
    assert all(torch.all(r.x == r.rid) for r in reqs)  # each got its own solution
    assert len([e for e in eng.events if e[0] == "release"]) == len(sizes)
    assert eng.free == budget and not eng.slots
    assert stats == {"iterations": eng.iters, "launches": 7 * eng.iters}
    # never more than the budget in use: replay the admissions and releases
    in_use, peak = 0, 0
    ids = {}
    for ev in eng.events:
        if ev[0] == "add":
            ids[len(ids)] = sizes[ev[1]] ** 3
            in_use += sizes[ev[1]] ** 3
            peak = max(peak, in_use)
        elif ev[0] == "release":
            in_use -= ids[ev[1]]
    assert peak <= budget


def test_request_larger_than_budget_is_refused(fake):
    reqs = requests([20])
    with pytest.raises(ValueError):
        serving.serve_continuous(reqs, 1000, max_slots=4, kmax=8)


def test_late_arrivals_wait_for_their_time(fake):
    reqs = requests([6, 6])
    reqs[1].arrival = 0.05
    serving.serve_continuous(reqs, 10 ** 4, max_slots=4, kmax=8, iters_per_tick=2)
    assert reqs[1].t_admit >= 0.05
    assert all(r.result["status"] == 0 for r in reqs)
