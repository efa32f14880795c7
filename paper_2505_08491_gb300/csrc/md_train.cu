// Training of the preconditioner network (placeholder entry points until the
// backward kernels land).
#include "md_internal.h"

extern "C" md_status md_cnn_backward(const md_cnn*, int, int, const float*, const float*, float*, float*, md_stream) {
    md_set_error("md_cnn_backward: not built yet");
    return MD_ERR_UNIMPLEMENTED;
}

extern "C" md_status md_train(md_cnn*, const md_train_cfg*) {
    md_set_error("md_train: not built yet");
    return MD_ERR_UNIMPLEMENTED;
}

extern "C" md_status md_train_loss(const md_cnn*, int, const md_op* const*, const float* const*, double*, float*,
                                   md_stream) {
    md_set_error("md_train_loss: not built yet");
    return MD_ERR_UNIMPLEMENTED;
}
