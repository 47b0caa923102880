"""GB300 (sm_103a) LIETS QSGS porous-media generator.

The generator runs in the CUDA library ``libqsgs`` (C ABI in include/qsgs.h);
``paper_2602_11734_gb300.qsgs`` is its Python binding.  Importing this
package loads nothing: the library is opened on first use and its absence
raises instead of falling back to the CPU.
"""

__all__ = ["qsgs", "workloads", "build"]
