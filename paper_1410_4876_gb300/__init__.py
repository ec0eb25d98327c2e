"""GB300 (sm_103a) enumeration of all chordless cycles (arXiv 1410.4876).

``paper_1410_4876_gb300.cc`` binds the C ABI of ``include/cc.h`` (the CUDA library in
``_build/libcc.so``, built by ``paper_1410_4876_gb300.build``); ``inputs`` holds the
seeded synthetic graph generators.  Submodules are imported on demand so that the
generators can be used without the CUDA library.
"""
__all__ = ["cc", "inputs", "build"]
