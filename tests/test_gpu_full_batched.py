"""The batched workload at its full size (1774 key+payload arrays, 2^28 keys
in one segmented call, the input bench.py times).  The oracle cannot sort
2^28 keys segment by segment in seconds, so the output is pinned by
properties that together determine it uniquely -- inside every segment the
keys ascend, every payload (= the key's input position) stays in its
segment and appears exactly once, each payload points at the key it carries,
and equal keys keep increasing payloads -- and sampled segments are compared
with the oracle exactly."""
import numpy as np
import pytest

import oracle
import synth
from tests._gpu import to_dev, to_host_u32, to_host_u64

pytestmark = pytest.mark.gpu
CHUNK = 1 << 25


def test_full_batched_workload():
    import torch
    import paper_cs_0004013_gb300 as rs
    keys, vals, offs = synth.segmented_batch(synth.CONFIG_SEED + 4)
    n, nseg = keys.size, offs.size - 1
    free, _ = torch.cuda.mem_get_info()
    if free < n * 4 * 6 + (2 << 30):
        pytest.skip("not enough free device memory")
    ko, vo, po = rs.sort_segmented(to_dev(keys), to_dev(vals), offs, num_parts=64)
    torch.cuda.synchronize()
    rs.rs_check_device_error()
    k = to_host_u32(ko)
    v = to_host_u32(vo)
    p = to_host_u64(po).reshape(nseg, 65)
    del ko, vo, po
    starts = offs[:-1].astype(np.int64)
    seg_of = np.repeat(np.arange(nseg, dtype=np.int32), np.diff(offs).astype(np.int64))
    seen = np.zeros(n, dtype=bool)
    for s in range(0, n, CHUNK):
        e = min(s + CHUNK, n)
        kk, vv, sg = k[s:e], v[s:e], seg_of[s:e]
        # each payload stays in its own segment and carries its own key
        assert np.all(vv >= starts[sg]) and np.all(vv < offs[1:][sg].astype(np.int64)), "payload left its segment"
        assert np.array_equal(keys[vv], kk), "payload does not point at its key"
        seen[vv] = True
        # ascending keys, and increasing payloads on equal keys, within a segment
        e1 = min(e + 1, n)
        nxt_k, nxt_v, nxt_s = k[s + 1:e1], v[s + 1:e1], seg_of[s + 1:e1]
        m = nxt_s == sg[: nxt_s.size]
        a, b = kk[: nxt_k.size][m], nxt_k[m]
        assert np.all(b >= a), "keys descend inside a segment"
        eq = b == a
        assert np.all(nxt_v[m][eq] > vv[: nxt_v.size][m][eq]), "equal keys lost their input order"
    assert seen.all(), "payloads are not a permutation"
    # partition offsets of every segment, and exact comparison on sampled segments
    for i in range(nseg):
        assert np.array_equal(p[i], oracle.partition_offsets(int(offs[i + 1] - offs[i]), 64) + offs[i])
    rng = np.random.default_rng(4)
    sizes = np.diff(offs)
    pick = set(rng.choice(nseg, 20, replace=False).tolist()) | {int(np.argmax(sizes)), int(np.argmin(sizes))}
    for i in sorted(pick):
        a, b = int(offs[i]), int(offs[i + 1])
        wk, wv = oracle.sort_pairs(keys[a:b], vals[a:b])
        assert np.array_equal(k[a:b], wk) and np.array_equal(v[a:b], wv), f"segment {i}"
