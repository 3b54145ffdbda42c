"""The end-to-end pipeline of bench.py (pack-from-host, compute and
unpack-to-host streams joined by events) gives, for every point, exactly the
result of the same point run alone on one stream: no operand is repacked
before the previous step's routine and unpack of that point are done."""
import pytest
import torch

import bench
import paper_1704_02457_gb300 as bf

pytestmark = pytest.mark.gpu

# more points than input and output slots, so both rings wrap within a step
SPEC = [("dpotrf_l", 16, 3000), ("dgemm_nt", 8, 5000), ("dsyrk_dpotrf_ln", 96, 300), ("dtrsm_rltn", 32, 900),
        ("dsyrk_ln", 4, 20000), ("dgemm_nt", 64, 400), ("dpotrf_l", 128, 200), ("dtrsm_rltn", 8, 7000),
        ("dsyrk_dpotrf_ln", 4, 30000)]


def test_e2e_pipeline_equals_each_point_run_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_02457_gb300.build import build
    build()
    bf.load()
    dev = torch.device("cuda")
    pts = [bench.Point(r, n, dev, seed=900 + i, batch=bt) for i, (r, n, bt) in enumerate(SPEC)]
    pipe = bench.E2EPipeline(pts, dev)
    assert len(pipe.plan) > pipe.NO
    outs = [torch.empty(p.batch * p.n * p.n, dtype=torch.float64, pin_memory=True) for p, _ in pipe.plan]
    pipe.step()
    pipe.step(outs)  # the second step's results land in one host buffer per point
    torch.cuda.synchronize()
    for (p, ins), out in zip(pipe.plan, outs):
        for name, h in ins:
            bf.pack(h.to(dev), getattr(p, name))
        p.run(torch.cuda.current_stream())
        ref = torch.empty(p.batch, p.n, p.n, dtype=torch.float64, device=dev)
        bf.unpack(p.D, ref)
        torch.cuda.synchronize()
        # bitwise: D's untouched upper triangle may hold any bit pattern
        assert torch.equal(out.view(torch.int64), ref.cpu().view(-1).view(torch.int64)), (p.routine, p.n)
