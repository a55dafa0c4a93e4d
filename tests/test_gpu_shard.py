"""The sort across ranks with its rank-local steps on the GPU (librsort's
kernels): two gloo ranks sharing cuda:0, each sorting its shard; the
exchanges go through host memory.  Against the oracle's sort of all keys
split into the equal partitions."""
import numpy as np
import pytest

import synth
from tests.test_shard import run_ranks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["uniform", "clustered", "uneven"])
def test_two_gloo_ranks_on_the_gpu(tmp_path, case):
    if case == "uniform":
        shards = [synth.uniform31(1 << 20, 1), synth.uniform31(1 << 20, 2)]
    elif case == "clustered":
        shards = [synth.tight_clusters(300_000, 3), synth.gauss_mix(200_000, 4)]
    else:
        shards = [synth.uniform31(123_457, 5) | (synth.uniform31(123_457, 6) << np.uint32(1)),
                  synth.few_distinct(10, 7)]
    run_ranks(shards, tmp_path, use_cuda=True)
