"""The product path has no CPU fallback: without the compiled library every
call fails loudly, and CPU tensors are refused rather than computed some
other way.  (CPU only: nothing here reaches a GPU.)"""
import os
import subprocess
import sys

import pytest

from conftest import ROOT


def test_missing_library_fails_loudly():
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import paper_2304_05669_gb300 as F\n"
        "try:\n"
        "    F._native.lib()\n"
        "except RuntimeError as e:\n"
        "    print('refused:', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(3)\n" % ROOT)
    env = dict(os.environ, FIPT_LIBRARY="/nonexistent/libfipt.so")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr)
    assert "not found" in r.stdout


def test_cpu_tensors_are_refused():
    torch = pytest.importorskip("torch")
    import paper_2304_05669_gb300 as F
    x = torch.zeros((4, 3))
    with pytest.raises(TypeError):
        F.Scene(x, torch.zeros((1, 3), dtype=torch.int32), torch.zeros((1, 3)), torch.zeros((1, 3)))
    with pytest.raises(TypeError):
        F.emitter_classify(torch.zeros(400), 100)
    with pytest.raises(TypeError):
        F.render_fwd(x, torch.zeros((4, 6, 3)), torch.zeros((4, 6, 3)), [0.1, 0.5], x,
                     torch.zeros(4), torch.zeros(4))
