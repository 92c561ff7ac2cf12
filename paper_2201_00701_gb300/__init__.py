"""GB300-native EmbedSOM projection: hand-written sm_103a CUDA kernels behind
a C ABI (include/esom.h), with a thin ctypes binding.

Paper: "Scalable semi-supervised dimensionality reduction with GPU-accelerated
EmbedSOM" (EmbedSOM projection, Section 3.1; GPU implementation, Section 4).
"""
from .binding import (EsomError, Projector, esom_create, esom_destroy, esom_device_status,
                      esom_get_config, esom_get_stats, esom_knn, esom_landmark_version, esom_last_error,
                      esom_project, esom_project_host, esom_set_landmark_chunk,
                      esom_set_landmarks, load)

__all__ = ["EsomError", "Projector", "esom_create", "esom_destroy", "esom_device_status",
           "esom_get_config", "esom_get_stats", "esom_knn", "esom_landmark_version", "esom_last_error",
           "esom_project", "esom_project_host", "esom_set_landmark_chunk",
           "esom_set_landmarks", "load"]
