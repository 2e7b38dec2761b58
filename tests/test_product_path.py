"""The product path (the package and bench.py's timed legs) never imports the
oracle: only the tests, the smoke check and bench.py's CPU-baseline and
reference legs may."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_package_and_bench_do_not_import_the_oracle():
    code = (
        "import sys; sys.argv = ['bench.py']\n"
        "import paper_2009_00083_gb300, paper_2009_00083_gb300.workloads, bench\n"
        "from tests.golden import store\n"
        "store.load_record('boxnoise3d_512'); store.load_authorized('boxnoise3d_512')\n"
        "store.load_set_authorized('mixed_batch_256'); store.load_set_authorized('serve_pool_16')\n"
        "print('oracle' in sys.modules)\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "False"
