"""The DAGS_CHECK build (libdags_check.so): index checks in the kernels pass
on valid inputs and report DAGS_E_BOUNDS, without faulting, when an input
holds an out-of-range index (an instance label past the region table)."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    from paper_2602_21644_gb300 import build, dags, synth
    dags.load(build.build(check=True))
    sc = synth.tiny_scene(0)
    cam = dags.Camera(*sc.camera.as_tuple())
    ctx = dags.Context(sc.records.shape[0], cam.width, cam.height, 1)
    gauss = torch.from_numpy(sc.records).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(sc.poses)).cuda()
    targets = torch.from_numpy(sc.targets).cuda()
    image, last, loss = ctx.forward(gauss, cam, poses, targets)
    ctx.backward(gauss, cam, poses, targets, image, last, dags.GRAD_GAUSS | dags.GRAD_POSE)
    torch.cuda.synchronize()
    ctx.check()
    P = cam.width * cam.height
    table = torch.tensor([[0.1, 0.05], [0.9, 0.8]], dtype=torch.float32, device="cuda")
    labels = torch.zeros(gauss.shape[0], dtype=torch.uint8, device="cuda")
    img = image[0].reshape(8, P).contiguous()
    inst = torch.zeros(P, dtype=torch.uint8, device="cuda")
    ctx.mp_update(gauss.clone(), cam, poses, targets, img, inst, table, labels)
    torch.cuda.synchronize()
    ctx.check()
    inst[P // 2] = 7                      # a label past the 2-row table
    ctx.mp_update(gauss.clone(), cam, poses, targets, img, inst, table, labels)
    torch.cuda.synchronize()
    try:
        ctx.check()
        print("NO-ERROR")
    except dags.DagsError as e:
        print("CODE", e.code)
    ctx.check()                           # cleared; the context stays usable
    ctx.forward(gauss, cam, poses, targets)
    torch.cuda.synchronize()
    ctx.check()
    print("OK")
""")


def test_check_build_detects_out_of_range_label():
    out = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT))], capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "CODE -7" in out.stdout and out.stdout.strip().endswith("OK"), out.stdout
