"""FP64 CPU oracle of the colour-gradient LBM step with the improved geometric wetting
scheme (arXiv 1707.00198, Sec. II).  Test infrastructure: imported only by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline legs; it never imports the
CUDA library and the CUDA library never imports it."""
from . import lbcg_oracle, observables  # noqa: F401
