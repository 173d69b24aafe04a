"""GB300-native MCQSG hot path: Metropolis sweeps + parallel tempering for the
2D +-J quantum Ising spin glass in Trotter-Suzuki form (Sec. 2.1 of "The QISG
suite"), behind the C ABI of ``include/qisg.h``."""
from .qisg import (Config, Instance, QisgError, QISG_LAYOUT_AUTO, QISG_LAYOUT_LANES,  # noqa: F401
                   QISG_LAYOUT_SAMPLES, ladder_linear, load, library_path)
