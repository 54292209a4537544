"""The tensor-core issue-path probe (mcl_probe_mma_rate): BF16 128 x 256 x 16
MMAs issued back to back from one thread run at 128 SM cycles each (4,096
multiply-accumulates per cycle per SM, the rate the MLP kernel's schedule is
measured against), and a group of G MMAs leaves only a third to a half of
them queued when the issuing thread moves on: a gap longer than that
between groups shows up in the time per group.  These are the two facts the kernel's issue
path is built on (operands computed before the gate, runs of landed
blocks)."""
import pytest

from gpu_helpers import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    return lib()


def test_back_to_back_mma_rate(M):
    clk, _ = M.probe_mma_rate(group=4, gap=0, n_groups=4000)
    print(f"\n{clk / 4:.2f} SM cycles per BF16 128x256x16 MMA")
    assert 126.0 <= clk / 4 <= 133.0


@pytest.mark.parametrize("group", [2, 4, 8])
def test_issue_run_ahead(M, group):
    """A gap far longer than the queued work costs its excess: the work
    left queued when the thread moved on is a fraction of the group's
    (the gap's clock reads are counted in it, so the estimate is low)."""
    work = 128.0 * group
    per_group, gap = M.probe_mma_rate(group=group, gap=64, n_groups=2000)
    queued = work - (per_group - gap)
    print(f"\nG={group}: gap {gap:.0f} clk -> {per_group:.0f} clk per group; queued ~{queued:.0f} clk "
          f"({queued / 128:.1f} MMAs)")
    assert per_group > gap
    assert 0.15 * work <= queued <= 0.75 * work


def test_short_gap_hidden_behind_a_large_group(M):
    """Eight MMAs leave about four queued: a short chain between groups
    costs nothing."""
    per_group, gap = M.probe_mma_rate(group=8, gap=2, n_groups=4000)
    assert gap < 0.4 * 1024
    assert per_group <= 1.03 * 1024, (per_group, gap)
