"""pilot_align_normal_eq_noalloc: the build-pass normal equations for callers that cannot
allocate device memory (an external pool owns it, or a latency-bound loop cannot risk an
allocation's implicit device synchronisation).  The entry point keeps its scratch in a
fixed file-scope device array and writes into a caller-provided device buffer.

Checked through the C-ABI against the handle-based pilot_align_debug_normal_eq on the
same inputs, on two calls in a row with different pose counts (the second call must not
see the first call's scratch), plus the size limits.  This file is named to be collected
last so that a run stopping at the first failure has run every other test first; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S

from gpu_support import assert_normal_eq_close, device_frame, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def noalloc(torch, opts, fa, level, T):
    T_dev = torch.as_tensor(np.ascontiguousarray(T, np.float64), device="cuda")
    out = torch.full((T.shape[0], 29), float("nan"), dtype=torch.float64, device="cuda")
    st = B.normal_eq_noalloc(opts, fa, level, T_dev, out)
    assert st == B.PILOT_OK, B.pilot_align_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_the_handle_entry_point_on_two_calls(torch):
    f = S.make_frame(S.config_reduced_frame(n_hyps=6), S.frame_seed(2, 700))
    opts = B.Options()
    solver = B.Solver(opts)
    rng = np.random.default_rng(0)
    calls = [np.vstack([f.T_gt[None, :], f.T_hyps]), f.T_hyps[rng.permutation(f.M)[:3]]]
    for call, T in enumerate(calls):
        fa = device_frame(f, T)
        for level in (0, 2):
            ref = solver.normal_eq(fa, level, T)
            got = noalloc(torch, opts, fa, level, T)
            assert np.all(np.isfinite(got))
            for m in range(T.shape[0]):
                assert_normal_eq_close(got[m], ref[m], what=f"call {call} level {level} pose {m}")
    solver.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    f = S.make_frame(S.config_reduced_frame(crop_side=20, n_hyps=2), 5)
    opts = B.Options()
    T = np.repeat(f.T_hyps[:1], 257, axis=0)
    fa = device_frame(f, T)
    T_dev = torch.as_tensor(T, device="cuda")
    out = torch.zeros((257, 29), dtype=torch.float64, device="cuda")
    assert B.normal_eq_noalloc(B.Options(max_hyps=512), fa, 0, T_dev, out) == B.PILOT_EINVAL
    assert "256" in B.pilot_align_last_error()
    host = B.FrameArgs(f, B.host_arrays(f), is_device=False)
    assert B.normal_eq_noalloc(opts, host, 0, T_dev[:2], out[:2]) == B.PILOT_EINVAL
    assert "device frame" in B.pilot_align_last_error()
