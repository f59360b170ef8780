"""Row shards for the row-sharded DROP (host-side bookkeeping, no GPU): every block's rows
are split into contiguous runs whose union over the ranks is the block, in order; the
package's shard_rows on a generated system and the benchmark's per-run generation give the
same shards."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("world", [1, 2, 3])
def test_shards_partition_every_block(world):
    from paper_1803_01112_gb300 import shard_rows
    import bench
    spec = synth.spec_scaled_3d(nx=20, ny=20, nz=2, n_hist=3_001, n_angles=10, n_blocks=4, seed=11)
    s = synth.generate(spec, np.float32)
    bp = s.block_ptr()
    shards = [shard_rows(s.row_ptr, s.col, s.val, s.b, bp, k, world) for k in range(world)]
    for t in range(len(bp) - 1):
        rows = []
        for rp, col, val, b, sbp in shards:
            for i in range(int(sbp[t]), int(sbp[t + 1])):
                rows.append((tuple(col[rp[i]:rp[i + 1]]), tuple(val[rp[i]:rp[i + 1]]), float(b[i])))
        want = [(tuple(s.col[s.row_ptr[i]:s.row_ptr[i + 1]]), tuple(s.val[s.row_ptr[i]:s.row_ptr[i + 1]]),
                 float(s.b[i])) for i in range(int(bp[t]), int(bp[t + 1]))]
        assert rows == want
    for k in range(world):
        rp, col, val, b, sbp, _ = bench.shard_system(spec, np.float32, k, world)
        erp, ecol, evl, eb, esbp = shards[k]
        np.testing.assert_array_equal(rp, erp)
        np.testing.assert_array_equal(col, ecol)
        np.testing.assert_array_equal(val, evl)
        np.testing.assert_array_equal(b, eb.astype(np.float32))
        np.testing.assert_array_equal(sbp, esbp)
