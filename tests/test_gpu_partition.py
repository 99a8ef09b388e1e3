"""Row blocks of the operators on the device (ssd_apply_rows): the blocks of
a split application, written into one output, are bit-identical to the whole
application in both precisions; ssd_points_order is the layout's
permutation; the partition driver without a process group is the whole
application."""
import numpy as np
import pytest

from oracle import quadrature as Q

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name", ["FP32C", "FP64"])
def test_row_blocks_equal_whole_application(gpu_ctx, prec_name):
    import torch
    import paper_2110_10749_gb300 as ssd
    from paper_2110_10749_gb300 import parallel as par
    prec = getattr(ssd, prec_name)
    h = 1 / 16
    p = Q.ellipsoid_points((1.0, 0.8, 0.6), h, center=(0.05, 0.0, 0.0))
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    n = P.n
    order = ssd.points_order(gpu_ctx, P)
    assert np.array_equal(np.sort(order), np.arange(n))
    rng = np.random.default_rng(9)
    g = torch.as_tensor(rng.normal(size=n), device="cuda")
    v = torch.as_tensor(rng.normal(size=(3, n)), device="cuda")
    whole = {ssd.OP_LAPLACE_SL: ssd.laplace_SL(gpu_ctx, P, 3 * h, g, prec),
             ssd.OP_LAPLACE_DL: ssd.laplace_DL(gpu_ctx, P, 3 * h, g, prec),
             ssd.OP_STOKES_SL: ssd.stokes_SL(gpu_ctx, P, 3 * h, 1.3, v, prec),
             ssd.OP_STOKES_DL: ssd.stokes_DL(gpu_ctx, P, 3 * h, v, prec)}
    for op, ref in whole.items():
        dens = g if op in (ssd.OP_LAPLACE_SL, ssd.OP_LAPLACE_DL) else v
        out = torch.full_like(dens, float("nan"))
        blocks = par.row_blocks(n, 3)
        for b, e in blocks:
            ssd.apply_rows(gpu_ctx, P, op, 3 * h, dens, b, e, mu=1.3, prec=prec, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), op
        # one block alone writes only its rows
        b, e = blocks[1]
        part = ssd.apply_rows(gpu_ctx, P, op, 3 * h, dens, b, e, mu=1.3, prec=prec)
        mask = np.zeros(n, dtype=bool)
        mask[order[b:e]] = True
        pc = part.cpu().numpy()
        assert np.array_equal(pc[..., mask], ref.cpu().numpy()[..., mask])
        assert not pc[..., ~mask].any()
    assert torch.equal(par.device_apply_sharded(gpu_ctx, P, ssd.OP_STOKES_DL, 3 * h, v, prec=prec),
                       whole[ssd.OP_STOKES_DL])
    with pytest.raises(ssd.SsdError):
        ssd.apply_rows(gpu_ctx, P, ssd.OP_LAPLACE_DL, 3 * h, g, 10, 10)
    with pytest.raises(ssd.SsdError):
        ssd.apply_rows(gpu_ctx, P, ssd.OP_LAPLACE_DL, 3 * h, g, 0, n + 1)
    P.release()
