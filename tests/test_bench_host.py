"""Host checks of bench.py's roofline inputs: the algorithmic bytes per update
of each step kernel, and the rule that the ncu DRAM traffic committed under
profiles/ is reported only while the kernel source it was taken on is
unchanged (a stale figure is reported as null)."""
import hashlib
import os
import re
import shutil

import bench


def test_algorithmic_bytes_per_update():
    # 2D: p^n, p^{n-1} read, p^{n+1} written, cc shared by the sample's nsg
    # supergathers; adjoint adds the snapshot, and cc and the accumulator
    # (read + write) are shared
    assert bench.bytes_per_update(5) == {"forward": 12.0 + 0.8, "adjoint": 16.0 + 2.4}
    assert bench.bytes_per_update(1) == {"forward": 16.0, "adjoint": 28.0}
    # 3D: one wavefield per CTA, or pair tiles sharing cc (and the accumulator)
    assert bench.bytes_per_update(4, 3) == {"forward": 16.0, "adjoint": 28.0}
    assert bench.bytes_per_update(4, 3, True, True) == {"forward": 14.0, "adjoint": 22.0}


def _key(ndim):
    src = "stencil3d.cu" if ndim == 3 else "stencil.cu"
    prof = "step3d_layered3d_traffic.md" if ndim == 3 else "step2d_thrust2d_traffic.md"
    txt = open(os.path.join(bench.ROOT, "profiles", prof)).read()
    m = re.search(r"traffic-key %s code-sha256=([0-9a-f]+) forward_bytes_per_update=([0-9.]+) "
                  r"adjoint_bytes_per_update=([0-9.]+)" % re.escape(src), txt)
    assert m, prof
    return src, m


def test_committed_traffic_follows_the_kernel_source():
    for ndim in (2, 3):
        src, m = _key(ndim)
        kd = "3d" if ndim == 3 else "2d"
        cur = bench.kernel_source_hash(src)
        fwd = bench.committed_traffic("step%s_kernel<FWD>" % kd, ndim)
        adj = bench.committed_traffic("step%s_kernel<ADJ>" % kd, ndim)
        if cur == m.group(1):
            assert fwd == float(m.group(2)) and adj == float(m.group(3))
            # a plausible DRAM figure: within 25 % of the algorithmic bytes
            alg = bench.bytes_per_update(4 if ndim == 3 else 5, ndim)
            assert 0.75 < fwd / alg["forward"] < 1.25 and 0.75 < adj / alg["adjoint"] < 1.25
        else:
            assert fwd is None and adj is None


def test_kernel_hash_ignores_comments_only():
    src = open(os.path.join(bench.ROOT, "paper_2512_12797_gb300", "csrc", "stencil3d.cu")).read()
    assert "//" in src
    h = hashlib.sha256(src.encode()).hexdigest()
    assert bench.kernel_source_hash("stencil3d.cu") != h  # not the file's own hash


def test_stale_traffic_is_null(tmp_path, monkeypatch):
    # a copy of the tree whose kernel code differs by one statement, and one
    # whose comments differ
    for d in ("profiles", os.path.join("paper_2512_12797_gb300", "csrc")):
        os.makedirs(tmp_path / d, exist_ok=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "step3d_layered3d_traffic.md"), tmp_path / "profiles")
    src = open(os.path.join(bench.ROOT, "paper_2512_12797_gb300", "csrc", "stencil3d.cu"), "rb").read()
    out = tmp_path / "paper_2512_12797_gb300" / "csrc" / "stencil3d.cu"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    out.write_bytes(src + b"\nstatic int changed_code;\n")
    assert bench.committed_traffic("step3d_kernel<FWD>", 3) is None
    out.write_bytes(src + b"\n// a comment\n\n")
    assert bench.committed_traffic("step3d_kernel<FWD>", 3) == float(_key(3)[1].group(2))
