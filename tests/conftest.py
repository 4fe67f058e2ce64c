import os
import sys

# The oracle's NumPy/SciPy calls are many small LU factorisations and
# products; OpenBLAS with one thread per core spends most of its time
# synchronising on those (a 256 x 256 complex LU took 25 ms with 8 threads
# against 2 ms with 1).  Four threads keep the large top-level merges
# parallel.  Set before NumPy is first imported; an explicit setting wins.
for _var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "4")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
