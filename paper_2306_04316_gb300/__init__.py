"""GB300-native ray-casting point-in-polygon classification (sm_103a CUDA behind a C ABI)."""
