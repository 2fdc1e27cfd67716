"""The checkpoint / recompute schedule of the autograd layer (host logic, no
GPU): a fake solver whose state buffers hold the time step they represent
records every call, so the test can check that the forward checkpoints the
start of every segment with one step() call per segment, and that the
backward runs exactly one adjoint step per time step, from the last to the
first, each from the state at its own time, after seeding from the final
state -- for segment lengths that divide the run, do not divide it, and
exceed it."""
import pytest

torch = pytest.importorskip("torch")

from paper_1202_6081_gb300 import autograd as AG  # noqa: E402


class FakeSolver:
    """State buffer = one float64 holding its time step; adjoint field = one
    float64 counting the adjoint steps applied to it."""

    def __init__(self):
        self.buf = torch.zeros(1, dtype=torch.float64)
        self.calls = []

    def current_buffer(self):
        return self.buf

    def step(self, n):
        self.calls.append(("step", n))
        self.buf += n

    def new_state_buffer(self):
        return torch.full((1,), -1.0, dtype=torch.float64)

    def step_into(self, src, dst):
        assert src.item() >= 0, "recomputed from an unset buffer"
        self.calls.append(("step_into", int(src.item())))
        dst.copy_(src + 1)

    def new_adjoint_field(self):
        return torch.full((1,), -1.0, dtype=torch.float64)

    def adjoint_step(self, f_t, lam_in, lam_out, gF):
        assert lam_in.item() >= 0, "adjoint step before the seed"
        self.calls.append(("adjoint", int(f_t.item())))
        lam_out.copy_(lam_in + 1)


@pytest.mark.parametrize("nsteps,every", [(30, 7), (28, 7), (20, 20), (21, 20), (5, 8), (1, 1),
                                          (1, 3), (9, 1)])
@pytest.mark.parametrize("two_rings", [True, False])
def test_checkpoints_and_adjoint_order(monkeypatch, nsteps, every, two_rings):
    """Both schedules: two rings (the next segment recomputed beside the
    current one's adjoint steps) and one ring (when a second does not fit)."""
    monkeypatch.setattr(AG, "_second_ring_fits", lambda ring: two_rings)
    S = FakeSolver()
    ckpts = AG._forward_with_checkpoints(S, nsteps, every)
    # forward: one step() call per segment, a checkpoint at every segment start
    nseg = (nsteps + every - 1) // every
    assert [c for c in S.calls if c[0] == "step"] == [
        ("step", min(every, nsteps - s * every)) for s in range(nseg)]
    assert [int(c.item()) for c in ckpts] == [s * every for s in range(nseg)]
    assert S.buf.item() == nsteps
    # backward
    S.calls.clear()
    seeded = []

    def seed(buf, lam):
        seeded.append(int(buf.item()))
        lam.fill_(0.0)

    lam0 = AG._backward_segments(S, nsteps, every, ckpts, seed, None)
    assert seeded == [nsteps], "the seed reads the final state once"
    adj = [c[1] for c in S.calls if c[0] == "adjoint"]
    assert adj == list(range(nsteps - 1, -1, -1)), "one adjoint step per step, last to first"
    assert lam0.item() == nsteps
    # recomputation: each segment from its checkpoint, the end state only in
    # the last segment (where it seeds the adjoint)
    rec = [c[1] for c in S.calls if c[0] == "step_into"]
    want = []
    for s in reversed(range(nseg)):
        t0, t1 = s * every, min(s * every + every, nsteps)
        want += list(range(t0, t1 if s == nseg - 1 else t1 - 1))
    assert rec == want
