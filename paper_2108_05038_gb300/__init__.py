"""GB300-native vertical-bitmap Eclat (frequent-itemset mining).

``paper_2108_05038_gb300.fim`` is the binding of the C ABI (include/fim.h);
``paper_2108_05038_gb300.synth`` generates seeded synthetic databases.
Importing the package loads nothing; the CUDA library is loaded by the first
call into ``fim``.
"""

__all__ = ["fim", "synth"]


def __getattr__(name):
    if name in __all__:
        import importlib

        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
