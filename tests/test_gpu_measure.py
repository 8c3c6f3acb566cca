"""The measurement entry points run and check their arguments (their numbers are bench.py's)."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu


def test_scan_rate_runs_and_rejects_bad_shapes():
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    t = datagen.fact_table(3_000_017, seed=5, cols=["date", "discount", "quantity"])
    T = tqp.TableRef([up(t[c]) for c in ("date", "discount", "quantity")])
    ctx = tqp.Context(0, 64 << 20)
    try:
        out = torch.zeros(1, dtype=torch.int64, device="cuda")
        for shape in ((1024, 2, 2), (2048, 3, 2), (4096, 2, 1), (4096, 3, 1)):
            tqp.tqp_measure_scan_rate(ctx, T, *shape, out)
            assert ctx.status() == 0
        assert int(out.item()) != 0
        for shape, status in (((1000, 2, 1), tqp.ERR_INVALID_ARG), ((1024, 5, 1), tqp.ERR_INVALID_ARG),
                              ((1024, 2, 3), tqp.ERR_INVALID_ARG), ((8192, 4, 2), tqp.ERR_UNSUPPORTED)):
            with pytest.raises(tqp.TqpError) as e:
                tqp.tqp_measure_scan_rate(ctx, T, *shape, out)
            assert e.value.status == status, shape
        S = tqp.TableRef([up(datagen.string_column(1000, seed=5))])
        with pytest.raises(tqp.TqpError) as e:
            tqp.tqp_measure_scan_rate(ctx, S, 1024, 2, 1, out)
        assert e.value.status == tqp.ERR_INVALID_ARG
    finally:
        ctx.close()
