"""libmemsynth: GB300-native non-gridding maximum-entropy image synthesis.

Importing the package does not load the CUDA library; ``memsynth`` does, and
fails loudly when it is missing.
"""
__all__ = ["memsynth", "synth"]
