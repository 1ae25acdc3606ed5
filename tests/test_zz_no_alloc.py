"""The occupancy refresh that allocates nothing (ia_update_occupancy_static).

It is meant for callers that cannot allocate device memory while they run, such
as code whose device memory belongs to another allocator or a frame loop that
must not pay for cudaMalloc's implicit synchronisation.  Its density scratch is a
fixed array inside the library, shared by every call, so the test checks two
calls in a row (two different poses, so stale contents would show) against the
allocating entry point, and that grids beyond the fixed size are refused.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import synthetic as S
from gpu_helpers import make_ctx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ia():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_10550_b300 as ia
    ia.lib()
    return ia


@pytest.mark.parametrize("config", ["tiny", "full"])
def test_static_scratch_matches_allocating_entry_point(ia, config):
    sc = S.make_scene(config, 0)
    table, mlp = S.make_field(sc, 0)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    poses = [S.make_pose(sc, i) for i in (3, 11)]
    ia.ia_set_pose(ctx, np.stack([p[0] for p in poses]), np.stack([p[1] for p in poses]))
    words = (sc.occ_res ** 3 + 31) // 32
    for pose in (0, 1):  # two calls in a row share the static scratch
        ref = torch.zeros(words, dtype=torch.int32, device="cuda")
        got = torch.full((words,), -1, dtype=torch.int32, device="cuda")
        ia.ia_update_occupancy(ctx, pose, ia.IA_OCC_POSE, None, ref)
        ia.ia_update_occupancy_static(ctx, pose, got)
        torch.cuda.synchronize()
        # occupancy bits are integer results: the tests require them bit-exact
        assert torch.equal(got, ref), f"pose {pose}"
        assert int(torch.count_nonzero(ref)) > 0
    ia.ia_destroy(ctx)


def test_static_scratch_rejects_grids_beyond_its_size(ia):
    sc = S.make_scene("tiny", 0)
    sc.occ_res = 96  # 96^3 cells do not fit the 64^3 static scratch
    table, mlp = S.make_field(sc, 0)
    ctx = make_ctx(ia, torch, sc, table, mlp)
    th, tr = S.make_pose(sc, 0)
    ia.ia_set_pose(ctx, th[None], tr[None])
    with pytest.raises(ia.IAError) as e:
        ia.ia_update_occupancy_static(ctx, 0)
    assert e.value.status == ia.IA_ERR_LIMIT
    assert "static scratch" in ia.ia_last_error(ctx)
    ia.ia_destroy(ctx)
