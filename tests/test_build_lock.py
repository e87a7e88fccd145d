"""Concurrent builds (one per rank of a multi-GPU run) do not clobber each
other: the first compiles, the others wait on the build lock and load the
same library."""
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_concurrent_builds_serialise_and_agree():
    from paper_1710_02812_gb300 import _build
    _build.build()
    lib = _build.LIB
    # make the library stale so both processes see work to do
    src = _build.sources()[0]
    t = time.time() + 1
    os.utime(src, (t, t))
    code = ("import sys; sys.path.insert(0, %r); from paper_1710_02812_gb300 import _build, hsvd; "
            "_build.build(); print(hsvd.lib().hsvd_tree_levels(7))" % ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True) for _ in range(2)]
    for p in procs:
        out, err = p.communicate(timeout=900)
        assert p.returncode == 0, err[-2000:]
        assert out.strip() == "3"
    assert os.path.getmtime(lib) >= os.path.getmtime(src)
    assert not os.path.exists(lib + ".tmp")
