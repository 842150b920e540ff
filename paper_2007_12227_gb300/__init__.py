"""GB300-native phase-space-conserving Vlasov step (Edelen & Webb, Sec. III).

The compute path is the C-ABI library ``libvlasov.so`` built from ``csrc/``;
``vlasov`` is its thin ctypes binding. Importing this package loads nothing.
"""
__all__ = ["inputs", "vlasov"]
