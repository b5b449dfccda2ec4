"""The tracker's two staging slots, and its saved state.  Frames uploaded from pinned host memory on
a copy stream into the slot the next frame will read, while the current frame
runs (the end-to-end form of the benchmark), give the same bits as enqueueing
every launch of every frame eagerly, and every (frame kind, slot) graph is
captured and replayed."""
import numpy as np
import pytest

from paper_1807_08271_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_08271_gb300.tracker import Tracker  # noqa: E402

N, KF = 46, 15      # keyframe switches at frames 15, 30, 45: slots 0, 1, 0


def test_side_stream_uploads_into_alternating_slots_equal_the_eager_run():
    seq = synth.render_sequence(2, n_frames=N)
    I_dev = torch.from_numpy(seq["I"]).cuda()
    W_dev = torch.from_numpy(seq["W"]).cuda()
    I_host = torch.from_numpy(seq["I"]).pin_memory()
    W_host = torch.from_numpy(seq["W"]).pin_memory()
    args = dict(levels=4, iters=(5, 5, 5, 10), kf_every=KF, max_frames=N)

    eager = Tracker(640, 480, seq["K"], graphs=False, **args)
    s = torch.cuda.Stream()
    for k in range(N):
        eager.step(I_dev[k], W_dev[k], s)
    torch.cuda.synchronize()

    trk = Tracker(640, 480, seq["K"], **args)
    stream, copy_stream = torch.cuda.Stream(), torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    with torch.cuda.stream(stream):
        trk.step(I_dev[0], W_dev[0], stream)
        slot = 0
        SI, SW = trk.staging(0)
        SI.copy_(I_host[1], non_blocking=True)
        SW.copy_(W_host[1], non_blocking=True)
        copied[0].record(stream)
        for k in range(1, N):
            gate = torch.cuda.Event()
            gate.record(stream)                   # frame k-1 no longer reads the other slot
            stream.wait_event(copied[slot])
            SI, SW = trk.staging(slot)
            trk.step(SI, SW, stream)
            if k + 1 < N:
                other = slot ^ 1
                copy_stream.wait_event(gate)
                with torch.cuda.stream(copy_stream):
                    OI, OW = trk.staging(other)
                    OI.copy_(I_host[k + 1], non_blocking=True)
                    OW.copy_(W_host[k + 1], non_blocking=True)
                    copied[other].record(copy_stream)
                slot = other
    torch.cuda.synchronize()
    assert set(trk._graph) == {(False, 0), (False, 1), (True, 0), (True, 1)}
    assert np.array_equal(trk.is_kf[:N], eager.is_kf[:N])
    assert np.array_equal(trk.results.cpu().numpy(), eager.results.cpu().numpy())
    for a, b in ((trk.I_kf, eager.I_kf), (trk.W_kf, eager.W_kf), (trk.C_kf, eager.C_kf)):
        assert torch.equal(a, b)


def test_saved_state_resumes_with_the_bits_of_an_uninterrupted_run(tmp_path):
    """Tracking 40 frames straight through, and tracking 23, saving the state,
    loading it into a new tracker and tracking the remaining 17 (across the switch
    at frame 30 of a 15-frame keyframe period), give the same bits."""
    n, cut = 40, 23
    seq = synth.render_sequence(3, n_frames=n)
    I = torch.from_numpy(seq["I"]).cuda()
    W = torch.from_numpy(seq["W"]).cuda()
    args = dict(levels=4, iters=(5, 5, 5, 10), kf_every=KF, max_frames=n)
    full = Tracker(640, 480, seq["K"], **args)
    for k in range(n):
        full.step(I[k], W[k])
    first = Tracker(640, 480, seq["K"], **args)
    for k in range(cut):
        first.step(I[k], W[k])
    path = str(tmp_path / "state.npz")
    first.save_state(path)
    second = Tracker(640, 480, seq["K"], **args)
    second.load_state(path)
    for k in range(cut, n):
        second.step(I[k], W[k])
    torch.cuda.synchronize()
    assert second.k == full.k == n
    assert np.array_equal(second.results.cpu().numpy(), full.results.cpu().numpy())
    for a, b in ((second.I_kf, full.I_kf), (second.W_kf, full.W_kf), (second.C_kf, full.C_kf)):
        assert torch.equal(a, b)
    assert np.array_equal(second.trajectory(), full.trajectory())
