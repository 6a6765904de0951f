"""GB300-native weighted random sampling with alias tables (arXiv 1903.00227).

Modules:

* ``wrs``       -- the Python binding of ``libwrs.so`` (the C ABI of
  ``include/wrs.h``): single tables built by the parallel split construction
  (``AliasTable``), batches of many tables (``AliasBatch``), two-level tables
  with output-sensitive sampling (``AliasTable2``), many-request sampling.
* ``serve``     -- a continuous-batching request server over resident tables.
* ``workloads`` -- seeded synthetic weights (uniform, permuted Zipf).

``wrs`` raises ImportError when the CUDA library has not been built
(``python -c "import __graft_entry__ as g; g.build()"``): there is no CPU
fallback.
"""
